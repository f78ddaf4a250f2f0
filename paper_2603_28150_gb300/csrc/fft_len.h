// Per-length launchers of the FFT stages. FftLen<R, P> is defined in
// fft_kernels.cuh and instantiated, a few lengths per file, by fft_*.cu; the
// stage dispatch in fft.cu sees only these declarations.
#pragma once
#include "pat_internal.h"

namespace pat {

template <typename R, int P>
struct FftLen {
  // stage i row pass: real rows of in -> half spectra T[s][kx][y]
  static cudaError_t row_r2c(const R* in, int64_t in_stride, int nx_in, int ny_in, cx<R>* T, int tstride,
                             int64_t tslice, int S, const cx<R>* tw, cudaStream_t st, Samp sm);
  // stage i column pass: T -> X[s][kx][ky] (or the slot layout with `slot`)
  static cudaError_t col_fwd(const cx<R>* T, int tstride, int64_t tslice, int n_in, int ncols, int S,
                             cx<R>* out, int64_t out_stride, const cx<R>* tw, cudaStream_t st,
                             const int* slot);
  // stage iii column pass: spectrum -> T, rows cropped to n_out
  static cudaError_t col_inv(const cx<R>* in, int64_t in_stride, int ncols, int S, cx<R>* T, int tstride,
                             int64_t tslice, int n_out, const cx<R>* tw, cudaStream_t st, const int* slot);
  // stage iii row pass: T -> real image (optionally minus `sub`, squares summed)
  static cudaError_t row_c2r(const cx<R>* T, int tstride, int64_t tslice, int nx_out, int ny_out, R* out,
                             int64_t out_stride, int S, const R* sub, double* partials, const cx<R>* tw,
                             cudaStream_t st, int* nblocks, Samp sm);
  // fused residual pass between H and H* (inverse row, r = S H x - y, forward row);
  // with `total` its last block also sums the FP64 partials (block counter `count`)
  static cudaError_t row_resid(cx<R>* T, int tstride, int64_t tslice, int nx, int ny, const R* y,
                               int64_t y_stride, int S, double* partials, double* total,
                               unsigned* count, const cx<R>* tw, cudaStream_t st, int* nblocks,
                               Samp sm);
  // stage iii row pass with the FISTA step in place of the gradient store
  static cudaError_t row_c2r_step(const cx<R>* T, int tstride, int64_t tslice, int nx, int ny,
                                  int64_t plane, int S, const FistaStep& f, const cx<R>* tw,
                                  cudaStream_t st);
};

#define PAT_P_SWITCH(PV, CALL)                           \
  switch (PV) {                                          \
    case 16: { constexpr int P_ = 16; return CALL; }     \
    case 24: { constexpr int P_ = 24; return CALL; }     \
    case 32: { constexpr int P_ = 32; return CALL; }     \
    case 48: { constexpr int P_ = 48; return CALL; }     \
    case 64: { constexpr int P_ = 64; return CALL; }     \
    case 96: { constexpr int P_ = 96; return CALL; }     \
    case 128: { constexpr int P_ = 128; return CALL; }   \
    case 192: { constexpr int P_ = 192; return CALL; }   \
    case 256: { constexpr int P_ = 256; return CALL; }   \
    case 384: { constexpr int P_ = 384; return CALL; }   \
    case 512: { constexpr int P_ = 512; return CALL; }   \
    case 768: { constexpr int P_ = 768; return CALL; }   \
    case 1024: { constexpr int P_ = 1024; return CALL; } \
    default: return cudaErrorInvalidValue;               \
  }

}  // namespace pat
