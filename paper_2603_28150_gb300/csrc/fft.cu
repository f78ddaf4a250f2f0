// Stage dispatch of the batched 2D real FFT (Sec. 3.2, Eq. 16 terms (i) and
// (iii)): picks the per-length launchers FftLen<R, P> (fft_len.h; kernels in
// fft_kernels.cuh, instantiated by the fft_*.cu files) for the plan's px and py.
#include "fft_len.h"
#include "pat_internal.h"

namespace pat {
namespace {

template <typename R>
cudaError_t spectrum_t(const Plan& p, const R* in, int64_t in_stride, int nx_in, int ny_in,
                       cx<R>* out, int64_t out_stride, int S, cudaStream_t st, Samp sm,
                       const int* slot) {
  const Layout& L = p.L;
  const int tstride = ny_in + (ny_in & 1);
  const int64_t tslice = (int64_t)(L.px / 2 + 1) * tstride;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  cudaError_t e;
  auto row = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.px, (FftLen<R, P_>::row_r2c(in, in_stride, nx_in, ny_in, T, tstride, tslice, S, twx, st,
                                        sm)))
  };
  if ((e = row()) != cudaSuccess) return e;
  auto col = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (FftLen<R, P_>::col_fwd(T, tstride, tslice, ny_in, L.px / 2 + 1, S, out, out_stride,
                                        twy, st, slot)))
  };
  return col();
}

template <typename R>
cudaError_t spectrum_rows_t(const Plan& p, const R* in, int64_t in_stride, int nx_in, int ny_in,
                            int S, cudaStream_t st) {
  const Layout& L = p.L;
  const int tstride = ny_in + (ny_in & 1);
  const int64_t tslice = (int64_t)(L.px / 2 + 1) * tstride;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  PAT_P_SWITCH(L.px, (FftLen<R, P_>::row_r2c(in, in_stride, nx_in, ny_in, T, tstride, tslice, S, twx, st,
                                      no_sampling())))
}

template <typename R>
cudaError_t spectrum_cols_t(const Plan& p, int ny_in, cx<R>* out, int64_t out_stride, int S,
                            cudaStream_t st, const int* slot) {
  const Layout& L = p.L;
  const int tstride = ny_in + (ny_in & 1);
  const int64_t tslice = (int64_t)(L.px / 2 + 1) * tstride;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  PAT_P_SWITCH(L.py, (FftLen<R, P_>::col_fwd(T, tstride, tslice, ny_in, L.px / 2 + 1, S, out, out_stride,
                                      twy, st, slot)))
}

template <typename R>
cudaError_t image_t(const Plan& p, const cx<R>* in, int64_t in_stride, R* out, int64_t out_stride,
                    int S, const R* sub, double* sumsq, cudaStream_t st, int groups,
                    double* group_sums, Samp sm, const int* slot) {
  const Layout& L = p.L;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  cudaError_t e;
  int nblocks = 0;
  const bool grouped = groups > 0 && group_sums != nullptr;
  double* partials = (sumsq || grouped) ? p.red : nullptr;
  auto col = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (FftLen<R, P_>::col_inv(in, in_stride, L.px / 2 + 1, S, T, L.tstride, L.tslice, L.ny,
                                        twy, st, slot)))
  };
  if ((e = col()) != cudaSuccess) return e;
  auto row = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.px, (FftLen<R, P_>::row_c2r(T, L.tstride, L.tslice, L.nx, L.ny, out, out_stride, S, sub,
                                        partials, twx, st, &nblocks, sm)))
  };
  if ((e = row()) != cudaSuccess) return e;
  // partials are slice-major, so each group of S / groups slices owns a
  // contiguous run of nblocks / groups partials
  if (grouped) return launch_group_sums(p.red, nblocks / groups, groups, group_sums, st);
  if (sumsq) return launch_partials_sum(p.red, nblocks, sumsq, st);
  return cudaSuccess;
}

// Spectra of H x -> spectra of the residual r = S H x - y (S the measurement
// operator, identity without sampling): column inverse pass into T, the fused
// residual row pass in place, column forward pass into out; ||r||^2 summed as
// image_t does.
template <typename R>
cudaError_t residual_t(const Plan& p, const cx<R>* in, int64_t in_stride, const R* y,
                       int64_t y_stride, int S, double* sumsq, cudaStream_t st, int groups,
                       double* group_sums, Samp sm, const int* slot, cx<R>* out,
                       int64_t out_stride) {
  const Layout& L = p.L;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  cudaError_t e;
  int nblocks = 0;
  const bool grouped = groups > 0 && group_sums != nullptr;
  double* partials = (sumsq || grouped) ? p.red : nullptr;
  auto col = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (FftLen<R, P_>::col_inv(in, in_stride, L.px / 2 + 1, S, T, L.tstride, L.tslice, L.ny,
                                        twy, st, slot)))
  };
  if ((e = col()) != cudaSuccess) return e;
  auto row = [&]() -> cudaError_t {
    // one sum (not per group): the pass's last block reduces the partials itself
    double* total = grouped ? nullptr : sumsq;
    unsigned* count = reinterpret_cast<unsigned*>(p.iter_dev + 2);
    PAT_P_SWITCH(L.px, (FftLen<R, P_>::row_resid(T, L.tstride, L.tslice, L.nx, L.ny, y, y_stride, S,
                                          partials, total, count, twx, st, &nblocks, sm)))
  };
  if ((e = row()) != cudaSuccess) return e;
  if (grouped && (e = launch_group_sums(p.red, nblocks / groups, groups, group_sums, st)) !=
                     cudaSuccess)
    return e;
  auto colf = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (FftLen<R, P_>::col_fwd(T, L.tstride, L.tslice, L.ny, L.px / 2 + 1, S, out,
                                        out_stride, twy, st, slot)))
  };
  return colf();
}

template <typename R>
cudaError_t image_step_t(const Plan& p, const cx<R>* in, int64_t in_stride, int S,
                         const FistaStep& f, cudaStream_t st, const int* slot) {
  const Layout& L = p.L;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  cudaError_t e;
  auto col = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (FftLen<R, P_>::col_inv(in, in_stride, L.px / 2 + 1, S, T, L.tstride, L.tslice, L.ny,
                                        twy, st, slot)))
  };
  if ((e = col()) != cudaSuccess) return e;
  const int64_t plane = (int64_t)L.ny * L.nx;
  auto row = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.px, (FftLen<R, P_>::row_c2r_step(T, L.tstride, L.tslice, L.nx, L.ny, plane, S, f, twx,
                                             st)))
  };
  return row();
}

}  // namespace

cudaError_t launch_spectrum_rows(const Plan& p, const void* in, int64_t in_stride, int nx_in,
                                 int ny_in, int S, cudaStream_t s) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return spectrum_rows_t<double>(p, static_cast<const double*>(in), in_stride, nx_in, ny_in, S, s);
  return spectrum_rows_t<float>(p, static_cast<const float*>(in), in_stride, nx_in, ny_in, S, s);
}

cudaError_t launch_spectrum_cols(const Plan& p, int ny_in, void* out, int64_t out_stride, int S,
                                 cudaStream_t s, const int* slot) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return spectrum_cols_t<double>(p, ny_in, static_cast<cx<double>*>(out), out_stride, S, s, slot);
  return spectrum_cols_t<float>(p, ny_in, static_cast<cx<float>*>(out), out_stride, S, s, slot);
}

cudaError_t launch_image_step(const Plan& p, const void* in, int64_t in_stride, int S,
                              const FistaStep& f, cudaStream_t s, const int* slot) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return image_step_t<double>(p, static_cast<const cx<double>*>(in), in_stride, S, f, s, slot);
  return image_step_t<float>(p, static_cast<const cx<float>*>(in), in_stride, S, f, s, slot);
}

cudaError_t launch_residual(const Plan& p, const void* in, int64_t in_stride, const void* y,
                            int64_t y_stride, int S, double* sumsq, cudaStream_t s, int groups,
                            double* group_sums, Samp sm, const int* slot, void* out,
                            int64_t out_stride) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return residual_t<double>(p, static_cast<const cx<double>*>(in), in_stride,
                              static_cast<const double*>(y), y_stride, S, sumsq, s, groups,
                              group_sums, sm, slot, static_cast<cx<double>*>(out), out_stride);
  return residual_t<float>(p, static_cast<const cx<float>*>(in), in_stride,
                           static_cast<const float*>(y), y_stride, S, sumsq, s, groups, group_sums,
                           sm, slot, static_cast<cx<float>*>(out), out_stride);
}

cudaError_t launch_spectrum(const Plan& p, const void* in, int64_t in_stride, int nx_in, int ny_in,
                            void* out, int64_t out_stride, int S, cudaStream_t s, Samp sm,
                            const int* slot) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return spectrum_t<double>(p, static_cast<const double*>(in), in_stride, nx_in, ny_in,
                              static_cast<cx<double>*>(out), out_stride, S, s, sm, slot);
  return spectrum_t<float>(p, static_cast<const float*>(in), in_stride, nx_in, ny_in,
                           static_cast<cx<float>*>(out), out_stride, S, s, sm, slot);
}

cudaError_t launch_image(const Plan& p, const void* in, int64_t in_stride, void* out,
                         int64_t out_stride, int S, const void* sub, double* sumsq,
                         cudaStream_t s, int groups, double* group_sums, Samp sm,
                         const int* slot) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return image_t<double>(p, static_cast<const cx<double>*>(in), in_stride,
                           static_cast<double*>(out), out_stride, S,
                           static_cast<const double*>(sub), sumsq, s, groups, group_sums, sm,
                           slot);
  return image_t<float>(p, static_cast<const cx<float>*>(in), in_stride, static_cast<float*>(out),
                        out_stride, S, static_cast<const float*>(sub), sumsq, s, groups,
                        group_sums, sm, slot);
}

}  // namespace pat
