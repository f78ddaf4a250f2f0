// FFT stage launchers, double precision, transform lengths 2^k in [16, 1024].
#include "fft_kernels.cuh"

namespace pat {
PAT_FFT_INSTANTIATE(double, 16)
PAT_FFT_INSTANTIATE(double, 32)
PAT_FFT_INSTANTIATE(double, 64)
PAT_FFT_INSTANTIATE(double, 128)
PAT_FFT_INSTANTIATE(double, 256)
PAT_FFT_INSTANTIATE(double, 512)
PAT_FFT_INSTANTIATE(double, 1024)
}  // namespace pat
