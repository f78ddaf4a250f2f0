// Batched 2D real FFT stages of the operator (Sec. 3.2, Eq. 16 terms (i) and (iii)).
//
// A P-point complex DFT runs as a Stockham auto-sort FFT (Govindaraju et al.,
// SC'08 formulation) over 2-3 passes of radix 8/16: each thread holds one
// radix-R butterfly in registers, multiplies by exp(-2 pi i r k / (Ns R))
// (twiddles from a host FP64 table staged in shared memory) and writes the
// R outputs to their sorted positions; vectors live in shared memory between
// passes. The 2D real transform of a zero-padded n x n slice is split in two
// kernels so every global access is contiguous:
//   row pass    two real rows packed as one complex row (a + i b), FFT over x,
//               untangled into the kx in [0, P/2] half spectra of both rows,
//               written transposed: T[s][kx][y]
//   column pass FFT over y of each kx column (only the n data rows are
//               non-zero), written as X[s][kx][ky] = the contraction's layout.
// The inverse runs the mirror image: column inverse FFT keeping the first n
// rows (crop), then a packed complex-to-real row inverse keeping the first n
// columns. No normalisation here: 1/(px py) is folded into the table.
#include "pat_internal.h"

namespace pat {
namespace {

constexpr int kThreads = 256;

template <int P>
struct RadixPlan;
template <> struct RadixPlan<16>   { static constexpr int NST = 1, R0 = 16, R1 = 1, R2 = 1, RMAX = 16; };
template <> struct RadixPlan<32>   { static constexpr int NST = 2, R0 = 8,  R1 = 4, R2 = 1, RMAX = 8; };
template <> struct RadixPlan<64>   { static constexpr int NST = 2, R0 = 8,  R1 = 8, R2 = 1, RMAX = 8; };
template <> struct RadixPlan<128>  { static constexpr int NST = 2, R0 = 16, R1 = 8, R2 = 1, RMAX = 16; };
template <> struct RadixPlan<256>  { static constexpr int NST = 2, R0 = 16, R1 = 16, R2 = 1, RMAX = 16; };
template <> struct RadixPlan<512>  { static constexpr int NST = 3, R0 = 8,  R1 = 8, R2 = 8, RMAX = 8; };
template <> struct RadixPlan<1024> { static constexpr int NST = 3, R0 = 16, R1 = 8, R2 = 8, RMAX = 16; };

template <int P>
struct Shape {
  static constexpr int TPV = P / RadixPlan<P>::RMAX;             // threads per vector
  static constexpr int VPB = kThreads / TPV;                      // vectors per block
  static constexpr int VSTR = P + P / 16;                         // padded vector stride
};

// One padding slot per 16 elements keeps the radix-16 scatter of the first
// pass (stride 16) free of shared-memory bank conflicts.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// exp(-2 pi i m / 16) for m in [0, 8) (conjugated for the inverse); m is a
// compile-time constant after unrolling, so the switch folds away.
template <typename R, bool INV>
__device__ __forceinline__ cx<R> mul_w16(cx<R> b, int m) {
  const R c1 = (R)0.92387953251128675613;  // cos(pi/8)
  const R s1 = (R)0.38268343236508977173;  // sin(pi/8)
  const R h = (R)0.70710678118654752440;   // sqrt(2)/2
  cx<R> w;
  switch (m) {
    case 0: return b;
    case 4: return INV ? mk<R>(-b.y, b.x) : mk<R>(b.y, -b.x);  // * (+-i)
    case 1: w = mk<R>(c1, -s1); break;
    case 2: w = mk<R>(h, -h); break;
    case 3: w = mk<R>(s1, -c1); break;
    case 5: w = mk<R>(-s1, -c1); break;
    case 6: w = mk<R>(-h, -h); break;
    default: w = mk<R>(-c1, -s1); break;
  }
  if (INV) w.y = -w.y;
  return cmul(b, w);
}

template <int N>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// Butterfly passes of span LEN, 2 LEN, ..., N (compile-time recursion keeps
// every register index constant).
template <typename R, int N, int LEN, bool INV>
__device__ __forceinline__ void dit_passes(cx<R>* a) {
#pragma unroll
  for (int i = 0; i < N; i += LEN) {
#pragma unroll
    for (int k = 0; k < LEN / 2; ++k) {
      cx<R> u = a[i + k];
      cx<R> t = mul_w16<R, INV>(a[i + k + LEN / 2], k * (16 / LEN));
      a[i + k] = cadd(u, t);
      a[i + k + LEN / 2] = csub(u, t);
    }
  }
  if constexpr (LEN < N) dit_passes<R, N, 2 * LEN, INV>(a);
}

// In-register N-point DFT (N = 2, 4, 8, 16): radix-2 decimation in time.
template <typename R, int N, bool INV>
__device__ __forceinline__ void dft_reg(cx<R>* a) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bitrev<N>(i);
    if (i < j) {
      cx<R> t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  dit_passes<R, N, 2, INV>(a);
}

// One Stockham pass of radix RAD over a vector of P points held in shared
// memory (`buf`, padded indexing); NS = product of the earlier radices.
template <typename R, int P, int RAD, int NS, bool INV>
__device__ __forceinline__ void stage(cx<R>* buf, const cx<R>* tw, int tid) {
  constexpr int TPV = Shape<P>::TPV;
  constexpr int NB = P / RAD;
  constexpr int PER = NB / TPV;
  cx<R> v[PER][RAD];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * TPV;
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[q][r] = buf[pidx(j + r * NB)];
    if (NS > 1) {
      const int k = j & (NS - 1);
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        cx<R> w = tw[(r * k * (P / (NS * RAD))) & (P - 1)];
        if (INV) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
    }
    dft_reg<R, RAD, INV>(v[q]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * TPV;
    const int k = j & (NS - 1);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) buf[pidx(base + r * NS)] = v[q][r];
  }
  __syncthreads();
}

template <typename R, int P, bool INV>
__device__ __forceinline__ void fft_all(cx<R>* buf, const cx<R>* tw, int tid) {
  using PL = RadixPlan<P>;
  stage<R, P, PL::R0, 1, INV>(buf, tw, tid);
  if constexpr (PL::NST >= 2) stage<R, P, PL::R1, PL::R0, INV>(buf, tw, tid);
  if constexpr (PL::NST >= 3) stage<R, P, PL::R2, PL::R0 * PL::R1, INV>(buf, tw, tid);
}

template <typename R, int P>
__device__ __forceinline__ cx<R>* setup_smem(const cx<R>* tw_g, cx<R>** tw_s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = tw_g[i];
  *tw_s = tw;
  return tw + P;
}

template <typename R, int P>
constexpr size_t smem_bytes() {
  return sizeof(cx<R>) * (size_t)(P + Shape<P>::VPB * Shape<P>::VSTR);
}

// Stage i, row pass: rows y0 = 2 pair, y0 + 1 of slice s packed as a + i b,
// zero-padded from nx_in to P, transformed; half spectra written to
// T[s][kx][y] for kx in [0, P/2].
template <typename R, int P>
__global__ void __launch_bounds__(kThreads) k_row_r2c(const R* __restrict__ in, int64_t in_stride,
                                                      int nx_in, int ny_in, cx<R>* __restrict__ T,
                                                      int tstride, int64_t tslice,
                                                      const cx<R>* __restrict__ tw_g) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t s = blockIdx.y;
  const int pair0 = blockIdx.x * SH::VPB;
  const R* src = in + s * in_stride;
  for (int i = threadIdx.x; i < SH::VPB * P; i += kThreads) {
    const int vv = i / P, x = i % P;
    const int y0 = 2 * (pair0 + vv);
    R a = 0, b = 0;
    if (x < nx_in) {
      if (y0 < ny_in) a = src[(int64_t)y0 * nx_in + x];
      if (y0 + 1 < ny_in) b = src[(int64_t)(y0 + 1) * nx_in + x];
    }
    bufs[vv * SH::VSTR + pidx(x)] = mk<R>(a, b);
  }
  __syncthreads();
  fft_all<R, P, false>(bufs + v * SH::VSTR, tw, tid);
  cx<R>* dst = T + s * tslice;
  for (int i = threadIdx.x; i < SH::VPB * (P / 2 + 1); i += kThreads) {
    const int vv = i % SH::VPB, kx = i / SH::VPB;
    const int y0 = 2 * (pair0 + vv);
    if (y0 >= ny_in) continue;
    const cx<R> Z = bufs[vv * SH::VSTR + pidx(kx)];
    const cx<R> Zm = bufs[vv * SH::VSTR + pidx((P - kx) & (P - 1))];
    // A = (Z + conj Zm) / 2 (row y0), B = (Z - conj Zm) / (2i) (row y0 + 1)
    const cx<R> A = mk<R>((R)0.5 * (Z.x + Zm.x), (R)0.5 * (Z.y - Zm.y));
    const cx<R> B = mk<R>((R)0.5 * (Z.y + Zm.y), (R)-0.5 * (Z.x - Zm.x));
    cx<R>* o = dst + (int64_t)kx * tstride + y0;
    o[0] = A;
    o[1] = B;  // tstride is even, so y0 + 1 < tstride
  }
}

// Stage i, column pass: T[s][kx][0..n_in) zero-padded to P, FFT over y,
// written to out[s][kx][0..P) (slice stride out_stride).
template <typename R, int P>
__global__ void __launch_bounds__(kThreads) k_col_fwd(const cx<R>* __restrict__ T, int tstride,
                                                      int64_t tslice, int n_in, int ncols,
                                                      int64_t nvec, cx<R>* __restrict__ out,
                                                      int64_t out_stride,
                                                      const cx<R>* __restrict__ tw_g) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t g0 = (int64_t)blockIdx.x * SH::VPB;
  for (int i = threadIdx.x; i < SH::VPB * P; i += kThreads) {
    const int vv = i / P, y = i % P;
    const int64_t g = g0 + vv;
    cx<R> a = mk<R>(0, 0);
    if (g < nvec && y < n_in) {
      const int64_t s = g / ncols, kx = g % ncols;
      a = T[s * tslice + kx * tstride + y];
    }
    bufs[vv * SH::VSTR + pidx(y)] = a;
  }
  __syncthreads();
  fft_all<R, P, false>(bufs + v * SH::VSTR, tw, tid);
  for (int i = threadIdx.x; i < SH::VPB * P; i += kThreads) {
    const int vv = i / P, y = i % P;
    const int64_t g = g0 + vv;
    if (g >= nvec) continue;
    const int64_t s = g / ncols, kx = g % ncols;
    out[s * out_stride + kx * P + y] = bufs[vv * SH::VSTR + pidx(y)];
  }
}

// Stage iii, column pass: in[s][kx][0..P) inverse FFT over ky, rows
// [0, n_out) kept (crop) into T[s][kx][y].
template <typename R, int P>
__global__ void __launch_bounds__(kThreads) k_col_inv(const cx<R>* __restrict__ in,
                                                      int64_t in_stride, int ncols, int64_t nvec,
                                                      cx<R>* __restrict__ T, int tstride,
                                                      int64_t tslice, int n_out,
                                                      const cx<R>* __restrict__ tw_g) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t g0 = (int64_t)blockIdx.x * SH::VPB;
  for (int i = threadIdx.x; i < SH::VPB * P; i += kThreads) {
    const int vv = i / P, y = i % P;
    const int64_t g = g0 + vv;
    cx<R> a = mk<R>(0, 0);
    if (g < nvec) {
      const int64_t s = g / ncols, kx = g % ncols;
      a = in[s * in_stride + kx * P + y];
    }
    bufs[vv * SH::VSTR + pidx(y)] = a;
  }
  __syncthreads();
  fft_all<R, P, true>(bufs + v * SH::VSTR, tw, tid);
  for (int i = threadIdx.x; i < SH::VPB * P; i += kThreads) {
    const int vv = i / P, y = i % P;
    const int64_t g = g0 + vv;
    if (g >= nvec || y >= n_out) continue;
    const int64_t s = g / ncols, kx = g % ncols;
    T[s * tslice + kx * tstride + y] = bufs[vv * SH::VSTR + pidx(y)];
  }
}

// Stage iii, row pass: half spectra A = T[s][kx][y0], B = T[s][kx][y0 + 1]
// of two real rows, packed as Z = A + iB with the Hermitian extension
// Z[P - kx] = conj(A) + i conj(B), inverse FFT over x; Re -> row y0,
// Im -> row y0 + 1, columns [0, nx_out) kept. With `sub`, writes
// image - sub and accumulates its squares (FP64) per block into partials.
template <typename R, int P>
__global__ void __launch_bounds__(kThreads) k_row_c2r(const cx<R>* __restrict__ T, int tstride,
                                                      int64_t tslice, int nx_out, int ny_out,
                                                      R* __restrict__ out, int64_t out_stride,
                                                      const R* __restrict__ sub,
                                                      double* __restrict__ partials,
                                                      const cx<R>* __restrict__ tw_g) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t s = blockIdx.y;
  const int pair0 = blockIdx.x * SH::VPB;
  const cx<R>* src = T + s * tslice;
  for (int i = threadIdx.x; i < SH::VPB * (P / 2 + 1); i += kThreads) {
    const int vv = i % SH::VPB, kx = i / SH::VPB;
    const int y0 = 2 * (pair0 + vv);
    cx<R> A = mk<R>(0, 0), B = mk<R>(0, 0);
    if (y0 < ny_out) {
      A = src[(int64_t)kx * tstride + y0];
      if (y0 + 1 < ny_out) B = src[(int64_t)kx * tstride + y0 + 1];
    }
    if (kx == 0 || kx == P / 2) {  // spectra of real rows: real at DC and Nyquist
      A.y = 0;
      B.y = 0;
    }
    cx<R>* b = bufs + vv * SH::VSTR;
    b[pidx(kx)] = mk<R>(A.x - B.y, A.y + B.x);
    if (kx > 0 && kx < P / 2) b[pidx(P - kx)] = mk<R>(A.x + B.y, B.x - A.y);
  }
  __syncthreads();
  fft_all<R, P, true>(bufs + v * SH::VSTR, tw, tid);
  R* dst = out + s * out_stride;
  const R* sb = sub ? sub + s * out_stride : nullptr;
  double acc = 0.0;
  for (int i = threadIdx.x; i < SH::VPB * nx_out; i += kThreads) {
    const int vv = i / nx_out, x = i % nx_out;
    const int y0 = 2 * (pair0 + vv);
    if (y0 >= ny_out) continue;
    const cx<R> z = bufs[vv * SH::VSTR + pidx(x)];
    R r0 = z.x, r1 = z.y;
    const int64_t o0 = (int64_t)y0 * nx_out + x, o1 = o0 + nx_out;
    if (sb) {
      r0 -= sb[o0];
      acc += (double)r0 * (double)r0;
    }
    dst[o0] = r0;
    if (y0 + 1 < ny_out) {
      if (sb) {
        r1 -= sb[o1];
        acc += (double)r1 * (double)r1;
      }
      dst[o1] = r1;
    }
  }
  if (partials) {
    // deterministic block sum: warp shuffle tree, then warp 0 over the warps
    __shared__ double wsum[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double w = threadIdx.x < kThreads / 32 ? wsum[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = w;
    }
  }
}

template <typename R, int P>
cudaError_t set_smem_attr(const void* fn) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<R, P>());
}

// ---- dispatch on the transform length ---------------------------------------
template <typename R, int P>
cudaError_t row_r2c(const R* in, int64_t in_stride, int nx_in, int ny_in, cx<R>* T, int tstride,
                    int64_t tslice, int S, const cx<R>* tw, cudaStream_t st) {
  using SH = Shape<P>;
  cudaError_t e = set_smem_attr<R, P>((const void*)k_row_r2c<R, P>);
  if (e != cudaSuccess) return e;
  const int pairs = (ny_in + 1) / 2;
  dim3 grid((pairs + SH::VPB - 1) / SH::VPB, S);
  k_row_r2c<R, P><<<grid, kThreads, smem_bytes<R, P>(), st>>>(in, in_stride, nx_in, ny_in, T,
                                                                tstride, tslice, tw);
  return cudaGetLastError();
}

template <typename R, int P>
cudaError_t col_fwd(const cx<R>* T, int tstride, int64_t tslice, int n_in, int ncols, int S,
                    cx<R>* out, int64_t out_stride, const cx<R>* tw, cudaStream_t st) {
  using SH = Shape<P>;
  cudaError_t e = set_smem_attr<R, P>((const void*)k_col_fwd<R, P>);
  if (e != cudaSuccess) return e;
  const int64_t nvec = (int64_t)S * ncols;
  const int64_t blocks = (nvec + SH::VPB - 1) / SH::VPB;
  k_col_fwd<R, P><<<(unsigned)blocks, kThreads, smem_bytes<R, P>(), st>>>(
      T, tstride, tslice, n_in, ncols, nvec, out, out_stride, tw);
  return cudaGetLastError();
}

template <typename R, int P>
cudaError_t col_inv(const cx<R>* in, int64_t in_stride, int ncols, int S, cx<R>* T, int tstride,
                    int64_t tslice, int n_out, const cx<R>* tw, cudaStream_t st) {
  using SH = Shape<P>;
  cudaError_t e = set_smem_attr<R, P>((const void*)k_col_inv<R, P>);
  if (e != cudaSuccess) return e;
  const int64_t nvec = (int64_t)S * ncols;
  const int64_t blocks = (nvec + SH::VPB - 1) / SH::VPB;
  k_col_inv<R, P><<<(unsigned)blocks, kThreads, smem_bytes<R, P>(), st>>>(
      in, in_stride, ncols, nvec, T, tstride, tslice, n_out, tw);
  return cudaGetLastError();
}

template <typename R, int P>
cudaError_t row_c2r(const cx<R>* T, int tstride, int64_t tslice, int nx_out, int ny_out, R* out,
                    int64_t out_stride, int S, const R* sub, double* partials, const cx<R>* tw,
                    cudaStream_t st, int* nblocks) {
  using SH = Shape<P>;
  cudaError_t e = set_smem_attr<R, P>((const void*)k_row_c2r<R, P>);
  if (e != cudaSuccess) return e;
  const int pairs = (ny_out + 1) / 2;
  dim3 grid((pairs + SH::VPB - 1) / SH::VPB, S);
  *nblocks = (int)(grid.x * grid.y);
  k_row_c2r<R, P><<<grid, kThreads, smem_bytes<R, P>(), st>>>(
      T, tstride, tslice, nx_out, ny_out, out, out_stride, sub, partials, tw);
  return cudaGetLastError();
}

#define PAT_P_SWITCH(PV, CALL)                         \
  switch (PV) {                                        \
    case 16: { constexpr int P_ = 16; return CALL; }   \
    case 32: { constexpr int P_ = 32; return CALL; }   \
    case 64: { constexpr int P_ = 64; return CALL; }   \
    case 128: { constexpr int P_ = 128; return CALL; } \
    case 256: { constexpr int P_ = 256; return CALL; } \
    case 512: { constexpr int P_ = 512; return CALL; } \
    case 1024: { constexpr int P_ = 1024; return CALL; } \
    default: return cudaErrorInvalidValue;             \
  }

template <typename R>
cudaError_t spectrum_t(const Plan& p, const R* in, int64_t in_stride, int nx_in, int ny_in,
                       cx<R>* out, int64_t out_stride, int S, cudaStream_t st) {
  const Layout& L = p.L;
  const int tstride = ny_in + (ny_in & 1);
  const int64_t tslice = (int64_t)(L.px / 2 + 1) * tstride;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  cudaError_t e;
  auto row = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.px, (row_r2c<R, P_>(in, in_stride, nx_in, ny_in, T, tstride, tslice, S, twx, st)))
  };
  if ((e = row()) != cudaSuccess) return e;
  auto col = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (col_fwd<R, P_>(T, tstride, tslice, ny_in, L.px / 2 + 1, S, out, out_stride,
                                        twy, st)))
  };
  return col();
}

template <typename R>
cudaError_t image_t(const Plan& p, const cx<R>* in, int64_t in_stride, R* out, int64_t out_stride,
                    int S, const R* sub, double* sumsq, cudaStream_t st) {
  const Layout& L = p.L;
  cx<R>* T = static_cast<cx<R>*>(p.T);
  const cx<R>* twx = static_cast<const cx<R>*>(p.twx);
  const cx<R>* twy = static_cast<const cx<R>*>(p.twy);
  cudaError_t e;
  auto col = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.py, (col_inv<R, P_>(in, in_stride, L.px / 2 + 1, S, T, L.tstride, L.tslice, L.ny,
                                        twy, st)))
  };
  if ((e = col()) != cudaSuccess) return e;
  int nblocks = 0;
  double* partials = sumsq ? p.red : nullptr;
  auto row = [&]() -> cudaError_t {
    PAT_P_SWITCH(L.px, (row_c2r<R, P_>(T, L.tstride, L.tslice, L.nx, L.ny, out, out_stride, S, sub,
                                        partials, twx, st, &nblocks)))
  };
  if ((e = row()) != cudaSuccess) return e;
  if (sumsq) {
    return launch_partials_sum(p.red, nblocks, sumsq, st);
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_spectrum(const Plan& p, const void* in, int64_t in_stride, int nx_in, int ny_in,
                            void* out, int64_t out_stride, int S, cudaStream_t s) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return spectrum_t<double>(p, static_cast<const double*>(in), in_stride, nx_in, ny_in,
                              static_cast<cx<double>*>(out), out_stride, S, s);
  return spectrum_t<float>(p, static_cast<const float*>(in), in_stride, nx_in, ny_in,
                           static_cast<cx<float>*>(out), out_stride, S, s);
}

cudaError_t launch_image(const Plan& p, const void* in, int64_t in_stride, void* out,
                         int64_t out_stride, int S, const void* sub, double* sumsq,
                         cudaStream_t s) {
  if (S <= 0) return cudaSuccess;
  if (p.L.fp64)
    return image_t<double>(p, static_cast<const cx<double>*>(in), in_stride,
                           static_cast<double*>(out), out_stride, S,
                           static_cast<const double*>(sub), sumsq, s);
  return image_t<float>(p, static_cast<const cx<float>*>(in), in_stride, static_cast<float*>(out),
                        out_stride, S, static_cast<const float*>(sub), sumsq, s);
}

}  // namespace pat
