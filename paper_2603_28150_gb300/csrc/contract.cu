// Fourier-domain multiply-accumulate of the operator (Sec. 3.2, Eq. 16 term (ii)):
//   forward  Y[b][t][k] = sum_z Hh[k][t][z] X[b][z][k]          (Eq. 7)
//   adjoint  Z[b][z][k] = sum_t conj(Hh[k][t][z]) D[b][t][k]    (Eq. 11)
// for every stored frequency bin k. The table is read exactly once per call,
// so both kernels are HBM-bound table streams (1 flop per table byte):
//   - a CTA owns 32 consecutive bins (one per lane); the table is stored
//     [k/32][t][z-group][lane][z in group] so every warp load is 32 x 16 B =
//     512 contiguous bytes, streamed with evict-first loads;
//   - forward: the CTA's X tile (all z of its 32 bins, VB volumes) sits in
//     shared memory; warps split the time samples and each thread produces
//     Y for one (bin, t);
//   - adjoint: warps split the z-groups, each thread keeps its Z partial sums
//     in registers while walking t; D comes through the read-only cache.
// Real tables (even kernels) store one float per (k, t, z): the real and
// imaginary parts of X are contracted by the same real coefficient.
#include <algorithm>

#include "pat_internal.h"

namespace pat {
namespace {

constexpr int kWarps = 8;

template <typename R, bool CPLX>
struct Elem;  // table element type and z per 16-byte group
template <> struct Elem<float, false>  { typedef float T; static constexpr int ZG = 4; };
template <> struct Elem<float, true>   { typedef cx<float> T; static constexpr int ZG = 2; };
template <> struct Elem<double, false> { typedef double T; static constexpr int ZG = 2; };
template <> struct Elem<double, true>  { typedef cx<double> T; static constexpr int ZG = 1; };

// Streamed (evict-first) 16-byte load of the table.
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }

// Read-only-cache load of one complex value.
__device__ __forceinline__ cx<float> ldg_cx(const cx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldg_cx(const cx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}

// Unpacks one 16-byte table group into ZG elements.
template <typename R, bool CPLX>
__device__ __forceinline__ void unpack(const typename vec16<R>::type& v,
                                       typename Elem<R, CPLX>::T* e);
template <> __device__ __forceinline__ void unpack<float, false>(const float4& v, float* e) {
  e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
}
template <> __device__ __forceinline__ void unpack<float, true>(const float4& v, cx<float>* e) {
  e[0] = mk<float>(v.x, v.y); e[1] = mk<float>(v.z, v.w);
}
template <> __device__ __forceinline__ void unpack<double, false>(const double2& v, double* e) {
  e[0] = v.x; e[1] = v.y;
}
template <> __device__ __forceinline__ void unpack<double, true>(const double2& v, cx<double>* e) {
  e[0] = mk<double>(v.x, v.y);
}

// acc += h x   (forward)   /   acc += conj(h) x   (adjoint)
template <typename R>
__device__ __forceinline__ void mac(cx<R>& acc, R h, cx<R> x) {
  acc.x = fma(h, x.x, acc.x);
  acc.y = fma(h, x.y, acc.y);
}
// Real coefficient times complex value in FP32 as one paired FMA
// (fma.rn.f32x2: each lane rounded once, as the scalar FMAs are).
__device__ __forceinline__ void mac(cx<float>& acc, float h, cx<float> x) {
  asm("{\n .reg .b64 rh, rx, ra;\n mov.b64 rh, {%2, %2};\n mov.b64 rx, {%3, %4};\n"
      " mov.b64 ra, {%0, %1};\n fma.rn.f32x2 ra, rh, rx, ra;\n mov.b64 {%0, %1}, ra;\n}"
      : "+f"(acc.x), "+f"(acc.y)
      : "f"(h), "f"(x.x), "f"(x.y));
}
template <typename R>
__device__ __forceinline__ void mac(cx<R>& acc, cx<R> h, cx<R> x) {
  acc.x = fma(h.x, x.x, acc.x);
  acc.x = fma(-h.y, x.y, acc.x);
  acc.y = fma(h.x, x.y, acc.y);
  acc.y = fma(h.y, x.x, acc.y);
}
template <typename R>
__device__ __forceinline__ void mac_conj(cx<R>& acc, R h, cx<R> x) {
  mac(acc, h, x);
}
template <typename R>
__device__ __forceinline__ void mac_conj(cx<R>& acc, cx<R> h, cx<R> x) {
  acc.x = fma(h.x, x.x, acc.x);
  acc.x = fma(h.y, x.y, acc.x);
  acc.y = fma(h.x, x.y, acc.y);
  acc.y = fma(-h.y, x.x, acc.y);
}

// grid (nkb, ceil(batch / VB)); block kWarps * 32; dynamic smem VB * nzg*ZG * 32 complex.
template <typename R, bool CPLX, int VB>
__global__ void __launch_bounds__(kWarps * 32)
    k_contract_fwd(const typename vec16<R>::type* __restrict__ table,
                   const cx<R>* __restrict__ X, cx<R>* __restrict__ Y, int nz, int nt, int nzg,
                   int64_t K, int64_t Kpad, int batch) {
  typedef typename vec16<R>::type V;
  typedef typename Elem<R, CPLX>::T E;
  constexpr int ZG = Elem<R, CPLX>::ZG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* xs = reinterpret_cast<cx<R>*>(smem_raw);  // [VB][nzg*ZG][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t kb = blockIdx.x;
  const int64_t k = kb * 32 + lane;
  const int b0 = blockIdx.y * VB;
  const int nzp = nzg * ZG;
  pdl_wait();
  for (int i = threadIdx.x; i < VB * nzp * 32; i += blockDim.x) {
    const int l = i & 31, z = (i >> 5) % nzp, v = (i >> 5) / nzp;
    const int64_t kk = kb * 32 + l;
    cx<R> a = mk<R>(0, 0);
    if (b0 + v < batch && z < nz && kk < K) a = X[((int64_t)(b0 + v) * nz + z) * Kpad + kk];
    xs[i] = a;
  }
  __syncthreads();
  const V* tb = table + (kb * nt) * (int64_t)nzg * 32 + lane;
  for (int t = warp; t < nt; t += kWarps) {
    cx<R> acc[VB];
#pragma unroll
    for (int v = 0; v < VB; ++v) acc[v] = mk<R>(0, 0);
    const V* hp = tb + (int64_t)t * nzg * 32;
#pragma unroll 4
    for (int g = 0; g < nzg; ++g) {
      E e[ZG];
      unpack<R, CPLX>(ld_stream(hp + g * 32), e);
#pragma unroll
      for (int q = 0; q < ZG; ++q) {
#pragma unroll
        for (int v = 0; v < VB; ++v) mac(acc[v], e[q], xs[(v * nzp + g * ZG + q) * 32 + lane]);
      }
    }
    if (k < K) {
#pragma unroll
      for (int v = 0; v < VB; ++v)
        if (b0 + v < batch) Y[((int64_t)(b0 + v) * nt + t) * Kpad + k] = acc[v];
    }
  }
}

// grid (nkb, ceil(batch / VB), z-chunks); block kWarps * 32. Warp w of z-chunk c
// owns the z-groups g = c * kWarps * GPW + w + j * kWarps, j < GPW. Single-
// volume float variants are held to 32 registers so 8 CTAs (all 64 warp slots)
// stay resident: the stream needs the warps more than the registers.
template <typename R, bool CPLX, int VB, int GPW>
__global__ void __launch_bounds__(kWarps * 32, (sizeof(R) == 4 && !CPLX && VB == 1 && GPW <= 2) ? 8 : 1)
    k_contract_adj(const typename vec16<R>::type* __restrict__ table,
                   const cx<R>* __restrict__ D, cx<R>* __restrict__ Z, int nz, int nt, int nzg,
                   int64_t K, int64_t Kpad, int batch) {
  typedef typename vec16<R>::type V;
  typedef typename Elem<R, CPLX>::T E;
  constexpr int ZG = Elem<R, CPLX>::ZG;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t kb = blockIdx.x;
  const int64_t k = kb * 32 + lane;
  const int b0 = blockIdx.y * VB;
  const int gbase = blockIdx.z * kWarps * GPW + warp;
  cx<R> acc[GPW][ZG][VB];
#pragma unroll
  for (int j = 0; j < GPW; ++j)
#pragma unroll
    for (int q = 0; q < ZG; ++q)
#pragma unroll
      for (int v = 0; v < VB; ++v) acc[j][q][v] = mk<R>(0, 0);
  const bool kok = k < K;
  const V* tb = table + (kb * nt) * (int64_t)nzg * 32 + lane;
  pdl_wait();
#pragma unroll 1
  for (int t = 0; t < nt; ++t) {
    cx<R> d[VB];
#pragma unroll
    for (int v = 0; v < VB; ++v)
      d[v] = (kok && b0 + v < batch) ? ldg_cx(&D[((int64_t)(b0 + v) * nt + t) * Kpad + k])
                                     : mk<R>(0, 0);
    const V* hp = tb + (int64_t)t * nzg * 32;
#pragma unroll
    for (int j = 0; j < GPW; ++j) {
      const int g = gbase + j * kWarps;
      if (g < nzg) {
        E e[ZG];
        unpack<R, CPLX>(ld_stream(hp + g * 32), e);
#pragma unroll
        for (int q = 0; q < ZG; ++q)
#pragma unroll
          for (int v = 0; v < VB; ++v) mac_conj(acc[j][q][v], e[q], d[v]);
      }
    }
  }
  if (!kok) return;
#pragma unroll
  for (int j = 0; j < GPW; ++j) {
    const int g = gbase + j * kWarps;
#pragma unroll
    for (int q = 0; q < ZG; ++q) {
      const int z = g * ZG + q;
      if (g < nzg && z < nz) {
#pragma unroll
        for (int v = 0; v < VB; ++v)
          if (b0 + v < batch) Z[((int64_t)(b0 + v) * nz + z) * Kpad + k] = acc[j][q][v];
      }
    }
  }
}

// ---- D4-folded real tables ----------------------------------------------------
// A CTA owns 32 representatives {|kx|, |ky|} (one per lane); the table row of
// a representative is read once and applied to each of its (up to 4) bins,
// whose bin indices come from `members` ([block][lane][4], -1 = absent). CTA j
// reads stored chunk chunk[j] of 32 rows (chunk j when `chunk` is NULL): with
// radial sharing the CTAs of one radius group read the same chunk at about
// the same time, so DRAM delivers it once and L2 serves the others. One
// volume per blockIdx.y; every volume streams the (folded) table once.
constexpr int kRT = 4;   // forward: time samples per register block
constexpr int kTC = 32;  // adjoint: time samples per shared D tile

// Forward: warp w takes the time blocks w, w + 8, ... of kRT samples; per
// z-group it loads kRT table float4s and the 4 members' X from shared memory.
__global__ void __launch_bounds__(kWarps * 32, 2)
    k_fold_fwd(const float4* __restrict__ table, const int4* __restrict__ members,
               const int* __restrict__ chunk, const cx<float>* __restrict__ X,
               cx<float>* __restrict__ Y, int nz, int nt, int nzg, int64_t Kpad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* xs = reinterpret_cast<cx<float>*>(smem_raw);  // [4][nzp][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ub = blockIdx.x;
  const int b = blockIdx.y, nzp = nzg * 4;
  const int4 mem = members[ub * 32 + lane];
  const int bins[4] = {mem.x, mem.y, mem.z, mem.w};
  const cx<float>* Xb = X + (int64_t)b * nz * Kpad;
  pdl_wait();
  for (int z = warp; z < nzp; z += kWarps) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
      xs[(m * nzp + z) * 32 + lane] =
          (bins[m] >= 0 && z < nz) ? Xb[(int64_t)z * Kpad + bins[m]] : mk<float>(0.f, 0.f);
  }
  __syncthreads();
  const int64_t cb = chunk ? chunk[ub] : ub;
  const float4* tb = table + cb * nt * (int64_t)nzg * 32 + lane;
  for (int t0 = warp * kRT; t0 < nt; t0 += kWarps * kRT) {
    cx<float> acc[kRT][4];
#pragma unroll
    for (int r = 0; r < kRT; ++r)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[r][m] = mk<float>(0.f, 0.f);
#pragma unroll 4
    for (int g = 0; g < nzg; ++g) {
      float hv[kRT][4];
#pragma unroll
      for (int r = 0; r < kRT; ++r) {
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t0 + r < nt) h = ld_stream(tb + ((int64_t)(t0 + r) * nzg + g) * 32);
        hv[r][0] = h.x;
        hv[r][1] = h.y;
        hv[r][2] = h.z;
        hv[r][3] = h.w;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        cx<float> x[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) x[m] = xs[(m * nzp + g * 4 + q) * 32 + lane];
#pragma unroll
        for (int r = 0; r < kRT; ++r)
#pragma unroll
          for (int m = 0; m < 4; ++m) mac(acc[r][m], hv[r][q], x[m]);
      }
    }
#pragma unroll
    for (int r = 0; r < kRT; ++r) {
      const int t = t0 + r;
      if (t >= nt) break;
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (bins[m] >= 0) Y[((int64_t)b * nt + t) * Kpad + bins[m]] = acc[r][m];
    }
  }
}

// Adjoint: warp w of z-chunk c owns z-groups c*8*GPW + w + j*8; the 4 members'
// D values of kTC samples are staged in shared memory and reused by all warps.
template <int GPW>
__global__ void __launch_bounds__(kWarps * 32, 2)
    k_fold_adj(const float4* __restrict__ table, const int4* __restrict__ members,
               const int* __restrict__ chunk, const cx<float>* __restrict__ D,
               cx<float>* __restrict__ Z, int nz, int nt, int nzg, int64_t Kpad) {
  __shared__ cx<float> ds[kTC][4][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ub = blockIdx.x;
  const int b = blockIdx.y;
  const int gbase = blockIdx.z * kWarps * GPW + warp;
  const int4 mem = members[ub * 32 + lane];
  const int bins[4] = {mem.x, mem.y, mem.z, mem.w};
  const cx<float>* Db = D + (int64_t)b * nt * Kpad;
  const int64_t cb = chunk ? chunk[ub] : ub;
  const float4* tb = table + cb * nt * (int64_t)nzg * 32 + lane;
  cx<float> acc[GPW][4][4];
#pragma unroll
  for (int j = 0; j < GPW; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[j][q][m] = mk<float>(0.f, 0.f);
  pdl_wait();
  for (int t0 = 0; t0 < nt; t0 += kTC) {
    __syncthreads();
    for (int tt = warp; tt < kTC; tt += kWarps) {
      const int t = t0 + tt;
#pragma unroll
      for (int m = 0; m < 4; ++m)
        ds[tt][m][lane] =
            (bins[m] >= 0 && t < nt) ? Db[(int64_t)t * Kpad + bins[m]] : mk<float>(0.f, 0.f);
    }
    __syncthreads();
    const int tn = min(kTC, nt - t0);
    // 8 samples per step: their GPW x 8 table loads are issued together
    for (int tt = 0; tt < tn; tt += 8) {
      float4 h[8][GPW];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int j = 0; j < GPW; ++j) {
          const int g = gbase + j * kWarps;
          h[r][j] = (g < nzg && tt + r < tn)
                        ? ld_stream(tb + ((int64_t)(t0 + tt + r) * nzg + g) * 32)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        cx<float> d[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) d[m] = ds[(tt + r) & (kTC - 1)][m][lane];
#pragma unroll
        for (int j = 0; j < GPW; ++j) {
          const float hq[4] = {h[r][j].x, h[r][j].y, h[r][j].z, h[r][j].w};
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) mac(acc[j][q][m], hq[q], d[m]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < GPW; ++j) {
    const int g = gbase + j * kWarps;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int z = g * 4 + q;
      if (g < nzg && z < nz) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (bins[m] >= 0) Z[((int64_t)b * nz + z) * Kpad + bins[m]] = acc[j][q][m];
      }
    }
  }
}

cudaError_t fold_fwd(const Plan& p, const void* X, void* Y, int batch, cudaStream_t s) {
  const Layout& L = p.L;
  const size_t smem = sizeof(cx<float>) * 4 * (size_t)L.nzg * 4 * 32;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_fold_fwd,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)L.nrb, (unsigned)batch);
  return launch_pdl(k_fold_fwd, grid, dim3(kWarps * 32), smem, s,
                    static_cast<const float4*>(p.table), reinterpret_cast<const int4*>(p.rb_members),
                    static_cast<const int*>(p.rb_chunk), static_cast<const cx<float>*>(X),
                    static_cast<cx<float>*>(Y), L.nz, L.nt, L.nzg, L.Kpad);
}

cudaError_t fold_adj(const Plan& p, const void* D, void* Z, int batch, cudaStream_t s) {
  const Layout& L = p.L;
  constexpr int GPW = 2;
  dim3 grid((unsigned)L.nrb, (unsigned)batch,
            (unsigned)((L.nzg + kWarps * GPW - 1) / (kWarps * GPW)));
  return launch_pdl(k_fold_adj<GPW>, grid, dim3(kWarps * 32), 0, s,
                    static_cast<const float4*>(p.table), reinterpret_cast<const int4*>(p.rb_members),
                    static_cast<const int*>(p.rb_chunk), static_cast<const cx<float>*>(D),
                    static_cast<cx<float>*>(Z), L.nz, L.nt, L.nzg, L.Kpad);
}

template <typename R, bool CPLX, int VB>
cudaError_t fwd_t(const Plan& p, const void* X, void* Y, int batch, cudaStream_t s) {
  const Layout& L = p.L;
  constexpr int ZG = Elem<R, CPLX>::ZG;
  const size_t smem = sizeof(cx<R>) * (size_t)VB * L.nzg * ZG * 32;
  auto fn = k_contract_fwd<R, CPLX, VB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)fn,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)L.nkb, (unsigned)((batch + VB - 1) / VB));
  return launch_pdl(fn, grid, dim3(kWarps * 32), smem, s,
                    static_cast<const typename vec16<R>::type*>(p.table),
                    static_cast<const cx<R>*>(X), static_cast<cx<R>*>(Y), L.nz, L.nt, L.nzg, L.K,
                    L.Kpad, batch);
}

template <typename R, bool CPLX, int VB, int GPW>
cudaError_t adj_launch(const Plan& p, const void* D, void* Z, int batch, cudaStream_t s) {
  const Layout& L = p.L;
  const int per_chunk = kWarps * GPW;
  dim3 grid((unsigned)L.nkb, (unsigned)((batch + VB - 1) / VB),
            (unsigned)((L.nzg + per_chunk - 1) / per_chunk));
  return launch_pdl(k_contract_adj<R, CPLX, VB, GPW>, grid, dim3(kWarps * 32), 0, s,
                    static_cast<const typename vec16<R>::type*>(p.table),
                    static_cast<const cx<R>*>(D), static_cast<cx<R>*>(Z), L.nz, L.nt, L.nzg, L.K,
                    L.Kpad, batch);
}

template <typename R, bool CPLX, int VB>
cudaError_t adj_t(const Plan& p, const void* D, void* Z, int batch, cudaStream_t s) {
  // z-groups per warp: enough to cover nzg in one chunk up to 4 per warp,
  // beyond that several z-chunks each re-read D (small) but not the table.
  const int nzg = p.L.nzg;
  if (nzg <= kWarps) return adj_launch<R, CPLX, VB, 1>(p, D, Z, batch, s);
  if (nzg <= 2 * kWarps) return adj_launch<R, CPLX, VB, 2>(p, D, Z, batch, s);
  return adj_launch<R, CPLX, VB, 4>(p, D, Z, batch, s);
}

// Volumes per table pass: the table is read once per ceil(batch / VB) group.
template <typename R, bool CPLX>
cudaError_t fwd_vb(const Plan& p, const void* X, void* Y, int batch, cudaStream_t s) {
  if (batch >= 4) return fwd_t<R, CPLX, 4>(p, X, Y, batch, s);
  if (batch >= 2) return fwd_t<R, CPLX, 2>(p, X, Y, batch, s);
  return fwd_t<R, CPLX, 1>(p, X, Y, batch, s);
}
template <typename R, bool CPLX>
cudaError_t adj_vb(const Plan& p, const void* D, void* Z, int batch, cudaStream_t s) {
  if (batch >= 4) return adj_t<R, CPLX, 4>(p, D, Z, batch, s);
  if (batch >= 2) return adj_t<R, CPLX, 2>(p, D, Z, batch, s);
  return adj_t<R, CPLX, 1>(p, D, Z, batch, s);
}

}  // namespace

__global__ void k_to_slots(const float2* __restrict__ in, float2* __restrict__ out,
                           const int* __restrict__ slot, int64_t K, int64_t Kpad, int64_t srow,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / K, k = i % K;
    out[r * srow + __ldg(slot + k)] = in[r * Kpad + k];
  }
}

__global__ void k_from_slots(const float2* __restrict__ in, float2* __restrict__ out,
                             const int* __restrict__ slot, int64_t K, int64_t Kpad, int64_t srow,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / K, k = i % K;
    out[r * Kpad + k] = in[r * srow + __ldg(slot + k)];
  }
}

cudaError_t launch_to_slots(const Plan& p, const void* in, void* out, int64_t S, cudaStream_t s) {
  const int64_t n = S * p.L.K;
  const int g = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  k_to_slots<<<g, 256, 0, s>>>(static_cast<const float2*>(in), static_cast<float2*>(out),
                               p.fold_slot, p.L.K, p.L.Kpad, slot_row(p.L), n);
  return cudaGetLastError();
}

cudaError_t launch_from_slots(const Plan& p, const void* in, void* out, int64_t S,
                              cudaStream_t s) {
  const int64_t n = S * p.L.K;
  const int g = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  k_from_slots<<<g, 256, 0, s>>>(static_cast<const float2*>(in), static_cast<float2*>(out),
                                 p.fold_slot, p.L.K, p.L.Kpad, slot_row(p.L), n);
  return cudaGetLastError();
}

cudaError_t launch_contract_fwd(const Plan& p, const void* X, void* Y, int batch, cudaStream_t s) {
  if (p.tc_fwd && p.tc_min_batch > 0 && batch >= p.tc_min_batch)
    return tc_contract(p, p.tc_fwd, p.tc_adj, X, Y, batch, false, p.tc_err, s);
  if (p.L.fold) return fold_fwd(p, X, Y, batch, s);
  if (p.L.fp64)
    return p.L.real ? fwd_vb<double, false>(p, X, Y, batch, s) : fwd_vb<double, true>(p, X, Y, batch, s);
  return p.L.real ? fwd_vb<float, false>(p, X, Y, batch, s) : fwd_vb<float, true>(p, X, Y, batch, s);
}

cudaError_t launch_contract_adj(const Plan& p, const void* D, void* Z, int batch, cudaStream_t s) {
  if (p.tc_adj && p.tc_min_batch > 0 && batch >= p.tc_min_batch)
    return tc_contract(p, p.tc_fwd, p.tc_adj, D, Z, batch, true, p.tc_err, s);
  if (p.L.fold) return fold_adj(p, D, Z, batch, s);
  if (p.L.fp64)
    return p.L.real ? adj_vb<double, false>(p, D, Z, batch, s) : adj_vb<double, true>(p, D, Z, batch, s);
  return p.L.real ? adj_vb<float, false>(p, D, Z, batch, s) : adj_vb<float, true>(p, D, Z, batch, s);
}

}  // namespace pat
