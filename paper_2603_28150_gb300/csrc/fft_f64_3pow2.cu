// FFT stage launchers, double precision, transform lengths 3 * 2^k in [24, 768].
#include "fft_kernels.cuh"

namespace pat {
PAT_FFT_INSTANTIATE(double, 24)
PAT_FFT_INSTANTIATE(double, 48)
PAT_FFT_INSTANTIATE(double, 96)
PAT_FFT_INSTANTIATE(double, 192)
PAT_FFT_INSTANTIATE(double, 384)
PAT_FFT_INSTANTIATE(double, 768)
}  // namespace pat
