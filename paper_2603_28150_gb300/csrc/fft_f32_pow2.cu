// FFT stage launchers, float precision, transform lengths 2^k in [16, 1024].
#include "fft_kernels.cuh"

namespace pat {
PAT_FFT_INSTANTIATE(float, 16)
PAT_FFT_INSTANTIATE(float, 32)
PAT_FFT_INSTANTIATE(float, 64)
PAT_FFT_INSTANTIATE(float, 128)
PAT_FFT_INSTANTIATE(float, 256)
PAT_FFT_INSTANTIATE(float, 512)
PAT_FFT_INSTANTIATE(float, 1024)
}  // namespace pat
