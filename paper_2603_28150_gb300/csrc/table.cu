// Plan-time construction of the resident spectral table (Sec. 3.2: the
// depth-indexed impulse-response library, stored once, applied every call).
//
// Sources:
//   spatial h[nz][nt][py][px]        -> 2D real FFT per (z, t) on the device
//   spectral Hh[nz][nt][py][px/2+1]  -> transposed to kx-major
//   k-space medium                   -> generated here from the exact periodic
//                                       solution of Eq. 1-2 (one point source,
//                                       recorded on the depth planes)
// Every value is scaled by 1/(px py) (the inverse FFT normalisation) and
// scattered into the blocked layout [k/32][t][z-group][lane][z in group].
// Pass 1 over a transformed source measures max |Hh| and max |Im Hh|; the
// real layout is chosen when Im is negligible (even kernels), pass 2 fills it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "pat_internal.h"

namespace pat {
namespace {

// Table element store: real tables keep only the real part.
template <typename RT, bool CPLX>
struct Store;
template <typename RT>
struct Store<RT, false> {
  __device__ static void put(void* table, int64_t idx, double re, double) {
    static_cast<RT*>(table)[idx] = (RT)re;
  }
};
template <typename RT>
struct Store<RT, true> {
  __device__ static void put(void* table, int64_t idx, double re, double im) {
    cx<RT> v;
    v.x = (RT)re;
    v.y = (RT)im;
    static_cast<cx<RT>*>(table)[idx] = v;
  }
};

__device__ __forceinline__ int64_t table_index(int64_t k, int t, int z, int nt, int nzg, int ZG) {
  const int64_t kb = k >> 5;
  const int lane = (int)(k & 31);
  const int zg = z / ZG, q = z % ZG;
  return (((kb * nt + t) * nzg + zg) * 32 + lane) * ZG + q;
}

// src: complex (RS) values for nt_chunk time samples of one depth plane z.
// rowmajor = 0: src[t][kx * py + ky] with slice stride sstride (FFT output)
// rowmajor = 1: src[t][ky][kx] with kx in [0, px/2] (R2C layout)
template <typename RS, typename RT, bool CPLX>
__global__ void k_scatter(const cx<RS>* __restrict__ src, int64_t sstride, int rowmajor, int px,
                          int py, int z, int t0, int nt_chunk, int nt, int nzg, int ZG,
                          double scale, void* table) {
  const int64_t K = (int64_t)(px / 2 + 1) * py;
  const int64_t n = K * nt_chunk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int tt = (int)(i / K);
    const int64_t k = i % K;
    const int kx = (int)(k / py), ky = (int)(k % py);
    const cx<RS> v = rowmajor ? src[tt * sstride + (int64_t)ky * (px / 2 + 1) + kx]
                              : src[tt * sstride + k];
    Store<RT, CPLX>::put(table, table_index(k, t0 + tt, z, nt, nzg, ZG), (double)v.x * scale,
                         (double)v.y * scale);
  }
}

// max |v|^2 and max |Im v| over the same source indexing, as ordered bit
// patterns of non-negative doubles (atomicMax on the integer image).
template <typename RS>
__global__ void k_stats(const cx<RS>* __restrict__ src, int64_t sstride, int rowmajor, int px,
                        int py, int nt_chunk, unsigned long long* out) {
  const int64_t K = (int64_t)(px / 2 + 1) * py;
  const int64_t n = K * nt_chunk;
  double m2 = 0.0, mi = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int tt = (int)(i / K);
    const int64_t k = i % K;
    const int kx = (int)(k / py), ky = (int)(k % py);
    const cx<RS> v = rowmajor ? src[tt * sstride + (int64_t)ky * (px / 2 + 1) + kx]
                              : src[tt * sstride + k];
    const double re = v.x, im = v.y;
    m2 = fmax(m2, re * re + im * im);
    mi = fmax(mi, fabs(im));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    mi = fmax(mi, __shfl_xor_sync(0xffffffffu, mi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(m2));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(mi));
  }
}

// ---- k-space library generator ---------------------------------------------
// One CTA per 32 bins (one per lane, the table's block). For each time sample
// t the CTA evaluates c_m = cos(c t dt |k_m|) for m in [0, mz/2] (|k_m| only
// depends on |kz|, so m and mz - m coincide), with the phase t * u_m (turns)
// taken modulo 1 in 64-bit fixed point so large arguments keep full accuracy,
// then contracts over m with W[m][j] = w_m cos(2 pi m (z0 + j) / mz) / (mz px py)
// (w_m = 1 at m = 0 and mz/2, else 2) from shared memory.
__global__ void k_kspace(int px, int py, int mz, int nz, int nt, int nzg, int ZG, int cplx,
                         const unsigned long long* __restrict__ u_fix,  // [K][mz/2+1] phase/sample
                         const float* __restrict__ W,                   // [mz/2+1][nz]
                         void* table, int64_t K) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = mz / 2 + 1;
  float* ws = reinterpret_cast<float*>(smem_raw);  // [M][nz]
  float* cs = ws + (size_t)M * nz;                  // [M][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * 32 + lane;
  for (int i = threadIdx.x; i < M * nz; i += blockDim.x) ws[i] = W[i];
  for (int t = 0; t < nt; ++t) {
    __syncthreads();
    for (int m = warp; m < M; m += nwarp) {
      float c = 0.f;
      if (k < K) {
        const unsigned long long ph = (unsigned long long)t * u_fix[k * M + m];  // mod 2^64
        const float turns = (float)(ph >> 40) * (1.0f / 16777216.0f);          // [0, 1)
        c = cospif(2.0f * turns);
      }
      cs[m * 32 + lane] = c;
    }
    __syncthreads();
    for (int j = warp; j < nz; j += nwarp) {
      float acc = 0.f;
      for (int m = 0; m < M; ++m) acc = fmaf(cs[m * 32 + lane], ws[m * nz + j], acc);
      if (k < K) {
        const int64_t idx = table_index(k, t, j, nt, nzg, ZG);
        if (cplx) {
          cx<float> v;
          v.x = acc;
          v.y = 0.f;
          static_cast<cx<float>*>(table)[idx] = v;
        } else {
          static_cast<float*>(table)[idx] = acc;
        }
      }
    }
  }
}

// max |T[ka[j]] - T[kb[j]]| over pairs of bins of a real blocked table, every
// (t, z) (bits of a non-negative double).
__global__ void k_pair_check(const float* __restrict__ table, const int* __restrict__ ka,
                             const int* __restrict__ kb, int64_t npairs, int nt, int nzg,
                             unsigned long long* out) {
  const int64_t n = npairs * nt * nzg * 4;
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i & 3);
    const int64_t r = i >> 2;
    const int g = (int)(r % nzg);
    const int t = (int)((r / nzg) % nt);
    const int64_t j = r / ((int64_t)nzg * nt);
    const int64_t k = ka[j], kr = kb[j];
    const float a = table[(((k >> 5) * nt + t) * nzg + g) * 128 + (k & 31) * 4 + q];
    const float b = table[(((kr >> 5) * nt + t) * nzg + g) * 128 + (kr & 31) * 4 + q];
    m = fmax(m, fabs((double)a - (double)b));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// folded row r = full[row_bin[r]] (zero where row_bin[r] < 0) for every
// (t, z-group), real tables.
__global__ void k_fold_gather(const float4* __restrict__ full, float4* __restrict__ folded,
                              const int* __restrict__ row_bin, int64_t rows, int nt, int nzg) {
  const int64_t n = rows * nt * nzg;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(i % nzg);
    const int t = (int)((i / nzg) % nt);
    const int64_t u = i / ((int64_t)nzg * nt);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t k = row_bin[u];
    if (k >= 0) v = full[(((k >> 5) * nt + t) * nzg + g) * 32 + (k & 31)];
    folded[(((u >> 5) * nt + t) * nzg + g) * 32 + (u & 31)] = v;
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename RT, bool CPLX>
cudaError_t scatter_launch(const void* src, bool src64, int64_t sstride, int rowmajor,
                           const Layout& L, int z, int t0, int ntc, double scale, void* table,
                           cudaStream_t s) {
  const int64_t n = L.K * ntc;
  if (src64)
    k_scatter<double, RT, CPLX><<<grid_for(n), 256, 0, s>>>(
        static_cast<const cx<double>*>(src), sstride, rowmajor, L.px, L.py, z, t0, ntc, L.nt,
        L.nzg, L.zg, scale, table);
  else
    k_scatter<float, RT, CPLX><<<grid_for(n), 256, 0, s>>>(
        static_cast<const cx<float>*>(src), sstride, rowmajor, L.px, L.py, z, t0, ntc, L.nt,
        L.nzg, L.zg, scale, table);
  return cudaGetLastError();
}

cudaError_t scatter_any(const void* src, bool src64, int64_t sstride, int rowmajor, const Layout& L,
                        int z, int t0, int ntc, double scale, void* table, cudaStream_t s) {
  if (L.fp64)
    return L.real ? scatter_launch<double, false>(src, src64, sstride, rowmajor, L, z, t0, ntc, scale, table, s)
                  : scatter_launch<double, true>(src, src64, sstride, rowmajor, L, z, t0, ntc, scale, table, s);
  return L.real ? scatter_launch<float, false>(src, src64, sstride, rowmajor, L, z, t0, ntc, scale, table, s)
                : scatter_launch<float, true>(src, src64, sstride, rowmajor, L, z, t0, ntc, scale, table, s);
}

std::vector<double> twiddles(int n) {
  std::vector<double> w(2 * (size_t)n);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    w[2 * k] = std::cos(-2.0 * pi * k / n);
    w[2 * k + 1] = std::sin(-2.0 * pi * k / n);
  }
  return w;
}

// Causal FIR along time of every scalar of the resident table, in place:
// a[t] = sum_{tau < nr, tau <= t} r[tau] a[t - tau] (FP64 sums), computed for
// t from nt - 1 down to 0 so every term still reads the unfiltered value. The
// blocked layout keeps, per table block, nt rows of `inner` scalars (real and
// imaginary parts alike: the response is real).
template <typename S>
__global__ void k_sensor_fir(S* __restrict__ table, int64_t blocks, int nt, int64_t inner,
                             const double* __restrict__ r, int nr) {
  const int64_t n = blocks * inner;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    S* a = table + (i / inner) * nt * inner + i % inner;
    for (int t = nt - 1; t >= 0; --t) {
      double acc = 0.0;
      const int m = nr < t + 1 ? nr : t + 1;
      for (int tau = 0; tau < m; ++tau) acc += r[tau] * (double)a[(int64_t)(t - tau) * inner];
      a[(int64_t)t * inner] = (S)acc;
    }
  }
}

}  // namespace

int apply_sensor_response(Plan& p, const double* r, int nr, cudaStream_t s) {
  const Layout& L = p.L;
  const int64_t blocks = L.fold ? L.nch : L.nkb;  // stored chunks of 32 rows
  const int64_t inner = (int64_t)L.nzg * 32 * 16 / (int64_t)L.rsize;
  double* rd = nullptr;
  PAT_CUDA(dev_alloc(&rd, sizeof(double) * nr));
  cudaError_t e = cudaMemcpyAsync(rd, r, sizeof(double) * nr, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const int g = grid_for(blocks * inner);
    if (L.fp64)
      k_sensor_fir<double><<<g, 256, 0, s>>>(static_cast<double*>(p.table), blocks, L.nt, inner,
                                             rd, nr);
    else
      k_sensor_fir<float><<<g, 256, 0, s>>>(static_cast<float*>(p.table), blocks, L.nt, inner, rd,
                                            nr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(rd);
  if (e != cudaSuccess) return cuda_fail(e, "applying the sensor response");
  return PAT_OK;
}

void fold_enumerate(int P, std::vector<int>& members, std::vector<int>& rep,
                    std::vector<int>& slot) {
  const int half = P / 2;
  const int64_t K = (int64_t)(half + 1) * P;
  members.clear();
  rep.assign((size_t)K, -1);
  slot.assign((size_t)K, -1);
  for (int a = 0; a <= half; ++a)
    for (int b = a; b <= half; ++b) {
      // bins (kx, ky) of the half spectrum with {kx, |ky|} = {a, b}
      const int cand[4][2] = {{a, b}, {a, (P - b) % P}, {b, a}, {b, (P - a) % P}};
      int out[4] = {-1, -1, -1, -1}, n = 0;
      for (auto& c : cand) {
        const int k = c[0] * P + c[1];
        bool dup = false;
        for (int i = 0; i < n; ++i) dup |= out[i] == k;
        if (!dup) out[n++] = k;
      }
      const int u = (int)(members.size() / 4);
      for (int i = 0; i < 4; ++i) {
        members.push_back(out[i]);
        if (out[i] >= 0) {
          rep[out[i]] = u;
          slot[out[i]] = 4 * u + i;
        }
      }
    }
}

static void radial_blocks(int P, const std::vector<int>& members, int64_t U, FoldBlocks& fb);

void fold_blocks(int P, const std::vector<int>& members, int64_t U, bool radial, FoldBlocks& fb) {
  if (radial) {
    radial_blocks(P, members, U, fb);
    if (fb.nch < (U + 31) / 32) return;
    // every group size pads its last chunk: on small grids sharing can store
    // more chunks than it saves, and then the identity layout is kept
  }
  fb = FoldBlocks();
  fb.nrb = fb.nch = (U + 31) / 32;
  fb.rb_rep.assign((size_t)fb.nrb * 32, -1);
  fb.row_rep.assign((size_t)fb.nch * 32, -1);
  fb.rep_row.assign((size_t)U, -1);
  fb.rb_chunk.resize((size_t)fb.nrb);
  for (int64_t j = 0; j < fb.nrb; ++j) fb.rb_chunk[j] = (int)j;
  for (int64_t u = 0; u < U; ++u) fb.rb_rep[u] = fb.row_rep[u] = fb.rep_row[u] = (int)u;
}

// Radial sharing: representatives of equal a^2 + b^2 at the same lane of
// consecutive blocks that read one chunk.
static void radial_blocks(int P, const std::vector<int>& members, int64_t U, FoldBlocks& fb) {
  fb = FoldBlocks();
  fb.rep_row.assign((size_t)U, -1);
  // representatives by radius a^2 + b^2 (a representative's own bin is a P + b)
  std::map<int64_t, std::vector<int>> by_radius;
  for (int64_t u = 0; u < U; ++u) {
    const int64_t a = members[4 * u] / P, b = members[4 * u] % P;
    by_radius[a * a + b * b].push_back((int)u);
  }
  // radii ordered by group size m, then radius; 32 radii of equal m per chunk,
  // read by m consecutive blocks (lane l of block j: the j-th representative
  // of the chunk's l-th radius)
  std::map<size_t, std::vector<const std::vector<int>*>> by_size;
  for (const auto& kv : by_radius) by_size[kv.second.size()].push_back(&kv.second);
  for (const auto& sv : by_size) {
    const size_t m = sv.first;
    const auto& radii = sv.second;
    for (size_t r0 = 0; r0 < radii.size(); r0 += 32) {
      const int64_t ch = fb.nch++;
      fb.row_rep.resize((size_t)fb.nch * 32, -1);
      fb.rb_rep.resize((size_t)(fb.nrb + (int64_t)m) * 32, -1);
      for (size_t j = 0; j < m; ++j) fb.rb_chunk.push_back((int)ch);
      for (size_t l = 0; l < 32 && r0 + l < radii.size(); ++l) {
        const std::vector<int>& reps = *radii[r0 + l];
        fb.row_rep[(size_t)ch * 32 + l] = reps[0];
        for (size_t j = 0; j < m; ++j) {
          fb.rb_rep[((size_t)fb.nrb + j) * 32 + l] = reps[j];
          fb.rep_row[reps[j]] = (int)(ch * 32 + (int64_t)l);
        }
      }
      fb.nrb += (int64_t)m;
    }
  }
}

int install_fold_blocks(Plan& p, const std::vector<int>& members, const FoldBlocks& fb) {
  Layout& L = p.L;
  const bool radial = fb.nch != fb.nrb;
  std::vector<int> rbm(fb.rb_rep.size() * 4, -1);
  for (size_t v = 0; v < fb.rb_rep.size(); ++v)
    if (fb.rb_rep[v] >= 0)
      for (int i = 0; i < 4; ++i) rbm[4 * v + i] = members[4 * (size_t)fb.rb_rep[v] + i];
  dev_free(p.rb_members);
  dev_free(p.rb_chunk);
  dev_free(p.rep_row);
  p.rb_members = p.rb_chunk = p.rep_row = nullptr;
  PAT_CUDA(dev_alloc(&p.rb_members, rbm.size() * sizeof(int)));
  PAT_CUDA(cudaMemcpy(p.rb_members, rbm.data(), rbm.size() * sizeof(int), cudaMemcpyHostToDevice));
  PAT_CUDA(dev_alloc(&p.rb_chunk, fb.rb_chunk.size() * sizeof(int)));
  PAT_CUDA(cudaMemcpy(p.rb_chunk, fb.rb_chunk.data(), fb.rb_chunk.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
  if (radial) {
    PAT_CUDA(dev_alloc(&p.rep_row, fb.rep_row.size() * sizeof(int)));
    PAT_CUDA(cudaMemcpy(p.rep_row, fb.rep_row.data(), fb.rep_row.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
  }
  L.nrb = fb.nrb;
  L.nch = fb.nch;
  L.radial = radial;
  return PAT_OK;
}

int build_fold_maps(Plan& p, std::vector<int>* members_out) {
  Layout& L = p.L;
  std::vector<int> members, rep, slot;
  fold_enumerate(L.px, members, rep, slot);
  L.U = (int64_t)members.size() / 4;
  L.Upad = (L.U + 31) / 32 * 32;
  L.nub = L.Upad / 32;
  members.resize((size_t)L.Upad * 4, -1);
  for (int64_t k = 0; k < L.K; ++k)
    if (rep[k] < 0) return fail(PAT_ERR_CUDA, "internal: a bin without representative");
  if (members_out) *members_out = members;
  PAT_CUDA(dev_alloc(&p.fold_slot, slot.size() * sizeof(int)));
  PAT_CUDA(cudaMemcpy(p.fold_slot, slot.data(), slot.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
  PAT_CUDA(dev_alloc(&p.fold_members, members.size() * sizeof(int)));
  PAT_CUDA(dev_alloc(&p.fold_rep, rep.size() * sizeof(int)));
  PAT_CUDA(cudaMemcpy(p.fold_members, members.data(), members.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
  PAT_CUDA(cudaMemcpy(p.fold_rep, rep.data(), rep.size() * sizeof(int), cudaMemcpyHostToDevice));
  return PAT_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int device_of(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

// max over pairs j and every (t, z) of |T[ka[j]] - T[kb[j]]| of the real
// blocked (per-bin) table p.table; synchronises `s`.
static int max_pair_deviation(Plan& p, const std::vector<int>& ka, const std::vector<int>& kb,
                              cudaStream_t s, double* out) {
  const Layout& L = p.L;
  const int64_t n = (int64_t)ka.size();
  int *a_d = nullptr, *b_d = nullptr;
  unsigned long long* dev_max = nullptr;
  cudaError_t e = dev_alloc(&a_d, ka.size() * sizeof(int));
  if (e == cudaSuccess) e = dev_alloc(&b_d, kb.size() * sizeof(int));
  if (e == cudaSuccess) e = dev_alloc(&dev_max, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(a_d, ka.data(), ka.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b_d, kb.data(), kb.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_max, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess && n > 0) {
    k_pair_check<<<grid_for(n * L.nt * L.nzg * 4), 256, 0, s>>>(
        static_cast<const float*>(p.table), a_d, b_d, n, L.nt, L.nzg, dev_max);
    e = cudaGetLastError();
  }
  unsigned long long hm = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, dev_max, sizeof(hm), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(a_d);
  dev_free(b_d);
  dev_free(dev_max);
  if (e != cudaSuccess) return cuda_fail(e, "checking the symmetry of the table");
  memcpy(out, &hm, 8);
  return PAT_OK;
}

int build_table_from_source(Plan& p, const void* table, pat_table_format fmt, bool force_complex,
                            bool allow_fold, bool allow_radial, cudaStream_t s) {
  Layout& L = p.L;
  const bool spatial = fmt == PAT_TABLE_SPATIAL_F64 || fmt == PAT_TABLE_SPATIAL_F32;
  const bool src64 = fmt == PAT_TABLE_SPATIAL_F64 || fmt == PAT_TABLE_SPECTRAL_C128;
  const bool on_dev = is_device_ptr(table);
  const int64_t plane_src = spatial ? (int64_t)L.px * L.py : (int64_t)L.py * (L.px / 2 + 1);
  const size_t esz_src = spatial ? (src64 ? 8 : 4) : (src64 ? 16 : 8);
  const size_t csz = src64 ? 16 : 8;  // complex size of the transform precision
  const int64_t Kfull = (int64_t)(L.px / 2 + 1) * L.py;

  // Time samples per chunk: source staging plus transform buffers stay
  // below ~1 GiB.
  const size_t per_t = plane_src * esz_src + (spatial ? (size_t)Kfull * csz * 2 : 0);
  const int ntc = (int)std::min<int64_t>(L.nt, std::max<int64_t>(1, (1ll << 30) / (int64_t)per_t));

  void *stage = nullptr, *spec = nullptr, *Tprep = nullptr, *twx = nullptr, *twy = nullptr;
  unsigned long long* stats = nullptr;
  auto cleanup = [&]() {
    dev_free(stage);
    dev_free(spec);
    dev_free(Tprep);
    dev_free(twx);
    dev_free(twy);
    dev_free(stats);
  };
#define PREP_CUDA(call)               \
  do {                                \
    cudaError_t e_ = (call);          \
    if (e_ != cudaSuccess) {          \
      int rc_ = cuda_fail(e_, #call); \
      cleanup();                      \
      return rc_;                     \
    }                                 \
  } while (0)

  if (!on_dev) PREP_CUDA(dev_alloc(&stage, (size_t)ntc * plane_src * esz_src));
  PREP_CUDA(dev_alloc(&stats, 2 * sizeof(unsigned long long)));
  PREP_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), s));

  // A transform-only view of the plan in the source precision: the same
  // grid with its own twiddles and intermediate buffer (all py rows).
  Plan prep;
  prep.L = L;
  prep.L.fp64 = src64;
  if (spatial) {
    PREP_CUDA(dev_alloc(&spec, (size_t)ntc * Kfull * csz));
    PREP_CUDA(dev_alloc(&Tprep, (size_t)ntc * (L.px / 2 + 1) * L.py * csz));
    std::vector<double> wx = twiddles(L.px), wy = twiddles(L.py);
    if (src64) {
      PREP_CUDA(dev_alloc(&twx, wx.size() * 8));
      PREP_CUDA(dev_alloc(&twy, wy.size() * 8));
      PREP_CUDA(cudaMemcpy(twx, wx.data(), wx.size() * 8, cudaMemcpyHostToDevice));
      PREP_CUDA(cudaMemcpy(twy, wy.data(), wy.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> fx(wx.begin(), wx.end()), fy(wy.begin(), wy.end());
      PREP_CUDA(dev_alloc(&twx, fx.size() * 4));
      PREP_CUDA(dev_alloc(&twy, fy.size() * 4));
      PREP_CUDA(cudaMemcpy(twx, fx.data(), fx.size() * 4, cudaMemcpyHostToDevice));
      PREP_CUDA(cudaMemcpy(twy, fy.data(), fy.size() * 4, cudaMemcpyHostToDevice));
    }
    prep.T = Tprep;
    prep.twx = twx;
    prep.twy = twy;
  }

  // Spectra of depth z, samples [t0, t0 + n): pointer, slice stride, layout.
  auto transform = [&](int z, int t0, int n, const void** out, int64_t* out_stride,
                       int* rowmajor) -> cudaError_t {
    const char* base = static_cast<const char*>(table) +
                       ((int64_t)z * L.nt + t0) * plane_src * (int64_t)esz_src;
    const void* src = base;
    if (!on_dev) {
      cudaError_t e = cudaMemcpyAsync(stage, base, (size_t)n * plane_src * esz_src,
                                      cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return e;
      src = stage;
    }
    if (!spatial) {
      *out = src;
      *out_stride = plane_src;
      *rowmajor = 1;
      return cudaSuccess;
    }
    *out = spec;
    *out_stride = Kfull;
    *rowmajor = 0;
    return launch_spectrum(prep, src, (int64_t)L.px * L.py, L.px, L.py, spec, Kfull, n, s);
  };

  // Pass 1: statistics of the whole library.
  for (int z = 0; z < L.nz; ++z)
    for (int t0 = 0; t0 < L.nt; t0 += ntc) {
      const int n = std::min(ntc, L.nt - t0);
      const void* src;
      int64_t sstride;
      int rowmajor;
      PREP_CUDA(transform(z, t0, n, &src, &sstride, &rowmajor));
      if (src64)
        k_stats<double><<<grid_for(Kfull * n), 256, 0, s>>>(
            static_cast<const cx<double>*>(src), sstride, rowmajor, L.px, L.py, n, stats);
      else
        k_stats<float><<<grid_for(Kfull * n), 256, 0, s>>>(
            static_cast<const cx<float>*>(src), sstride, rowmajor, L.px, L.py, n, stats);
      PREP_CUDA(cudaGetLastError());
    }
  unsigned long long hs[2];
  PREP_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
  PREP_CUDA(cudaStreamSynchronize(s));
  double m2, mi;
  memcpy(&m2, &hs[0], 8);
  memcpy(&mi, &hs[1], 8);
  p.table_max_abs = std::sqrt(m2);
  p.table_max_imag = mi;
  set_representation(L, !force_complex && mi <= 1e-6 * p.table_max_abs);

  // Pass 2: fill the resident table.
  PREP_CUDA(dev_alloc(&p.table, L.table_bytes));
  PREP_CUDA(cudaMemsetAsync(p.table, 0, L.table_bytes, s));
  const double scale = 1.0 / ((double)L.px * (double)L.py);
  for (int z = 0; z < L.nz; ++z)
    for (int t0 = 0; t0 < L.nt; t0 += ntc) {
      const int n = std::min(ntc, L.nt - t0);
      const void* src;
      int64_t sstride;
      int rowmajor;
      PREP_CUDA(transform(z, t0, n, &src, &sstride, &rowmajor));
      PREP_CUDA(scatter_any(src, src64, sstride, rowmajor, L, z, t0, n, scale, p.table, s));
    }
  PREP_CUDA(cudaStreamSynchronize(s));
  cleanup();

  // D4 folding when every bin equals its representative (to 1e-6 of max |Hh|),
  // then radial sharing when every representative also equals the first
  // representative of its radius (same bound).
  if (allow_fold && fold_possible(L)) {
    std::vector<int> members;
    int rc = build_fold_maps(p, &members);
    if (rc != PAT_OK) return rc;
    const double tol = 1e-6 * p.table_max_abs / ((double)L.px * (double)L.py);
    std::vector<int> ka((size_t)L.K), kb((size_t)L.K);
    {
      std::vector<int> mem, repk, slot;
      fold_enumerate(L.px, mem, repk, slot);
      for (int64_t k = 0; k < L.K; ++k) {
        ka[k] = (int)k;
        kb[k] = mem[4 * (size_t)repk[k]];  // the representative's own bin
      }
    }
    double dmax = 0;
    if ((rc = max_pair_deviation(p, ka, kb, s, &dmax)) != PAT_OK) return rc;
    p.fold_deviation = dmax;
    if (dmax <= tol) {
      FoldBlocks fb;
      bool radial = false;
      if (allow_radial) {
        fold_blocks(L.px, members, L.U, true, fb);
        std::vector<int> ua((size_t)L.U), ub((size_t)L.U);
        for (int64_t u = 0; u < L.U; ++u) {
          ua[u] = members[4 * u];
          ub[u] = members[4 * (size_t)fb.row_rep[fb.rep_row[u]]];
        }
        double rmax = 0;
        if ((rc = max_pair_deviation(p, ua, ub, s, &rmax)) != PAT_OK) return rc;
        p.radial_deviation = rmax;
        radial = rmax <= tol;
      }
      if (!radial) fold_blocks(L.px, members, L.U, false, fb);
      if ((rc = install_fold_blocks(p, members, fb)) != PAT_OK) return rc;
      Layout F = L;
      set_representation(F, true, true);
      std::vector<int> row_bin(fb.row_rep.size(), -1);
      for (size_t r = 0; r < row_bin.size(); ++r)
        if (fb.row_rep[r] >= 0) row_bin[r] = members[4 * (size_t)fb.row_rep[r]];
      void* folded = nullptr;
      int* row_bin_d = nullptr;
      cudaError_t e = dev_alloc(&folded, F.table_bytes);
      if (e == cudaSuccess) e = dev_alloc(&row_bin_d, row_bin.size() * sizeof(int));
      if (e == cudaSuccess)
        e = cudaMemcpy(row_bin_d, row_bin.data(), row_bin.size() * sizeof(int),
                       cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        const int64_t rows = (int64_t)row_bin.size();
        k_fold_gather<<<grid_for(rows * F.nt * F.nzg), 256, 0, s>>>(
            static_cast<const float4*>(p.table), static_cast<float4*>(folded), row_bin_d, rows,
            F.nt, F.nzg);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      dev_free(row_bin_d);
      if (e != cudaSuccess) {
        dev_free(folded);
        return cuda_fail(e, "folding the table");
      }
      dev_free(p.table);
      p.table = folded;
      L = F;
    } else {
      dev_free(p.fold_members);
      dev_free(p.fold_rep);
      dev_free(p.fold_slot);
      p.fold_members = p.fold_rep = p.fold_slot = nullptr;
    }
  }
  return PAT_OK;
#undef PREP_CUDA
}

int build_table_kspace(Plan& p, const pat_medium& m, bool force_complex, bool allow_fold,
                       bool allow_radial, cudaStream_t s) {
  Layout& L = p.L;
  if (L.fp64) return fail(PAT_ERR_UNSUPPORTED, "k-space generation builds single-precision tables");
  set_representation(L, !force_complex);
  // |k| depends on kx^2 + ky^2 only, so with dx = dy on a square grid the
  // library is exactly D4-symmetric, and representatives of equal kx^2 + ky^2
  // have equal spectra: generate one row per stored row (per representative,
  // or with radial sharing per radius).
  std::vector<int> bins;
  if (kspace_folds(L, m, allow_fold)) {
    std::vector<int> members;
    int rc = build_fold_maps(p, &members);
    if (rc != PAT_OK) return rc;
    FoldBlocks fb;
    fold_blocks(L.px, members, L.U, allow_radial, fb);
    if ((rc = install_fold_blocks(p, members, fb)) != PAT_OK) return rc;
    set_representation(L, true, true);
    // unused rows (no representative) repeat the spectra of representative 0
    bins.resize(fb.row_rep.size());
    for (size_t r = 0; r < bins.size(); ++r)
      bins[r] = members[4 * (size_t)std::max(fb.row_rep[r], 0)];
  } else {
    bins.resize((size_t)L.K);
    for (int64_t k = 0; k < L.K; ++k) bins[k] = (int)k;
  }
  return kspace_generate(p, m, bins, s);
}

bool kspace_folds(const Layout& L, const pat_medium& m, bool allow_fold) {
  return allow_fold && fold_possible(L) && m.dx == m.dy;
}

int kspace_generate(Plan& p, const pat_medium& m, const std::vector<int>& bins, cudaStream_t s) {
  const Layout& L = p.L;
  const int64_t npos = (int64_t)bins.size();
  const int M = m.mz / 2 + 1;
  const double pi = 3.14159265358979323846;
  // u_m(k) = c dt |k_m| / (2 pi) turns per sample, as 64-bit fixed-point fractions.
  std::vector<unsigned long long> u((size_t)npos * M);
  for (int64_t pos = 0; pos < npos; ++pos) {
    const int64_t k = bins[pos];
    const int kx = (int)(k / L.py), kyi = (int)(k % L.py);
    const int ky = kyi < L.py / 2 ? kyi : kyi - L.py;
    const double wx = 2.0 * pi * kx / (L.px * m.dx), wy = 2.0 * pi * ky / (L.py * m.dy);
    for (int mm = 0; mm < M; ++mm) {
      const double wz = 2.0 * pi * mm / (m.mz * m.dz);
      const double turns = m.c * m.dt * std::sqrt(wx * wx + wy * wy + wz * wz) / (2.0 * pi);
      const double frac = turns - std::floor(turns);
      u[(size_t)pos * M + mm] = (unsigned long long)std::ldexp(frac, 64);
    }
  }
  std::vector<float> W((size_t)M * L.nz);
  const double scale = 1.0 / ((double)m.mz * L.px * L.py);
  for (int mm = 0; mm < M; ++mm)
    for (int j = 0; j < L.nz; ++j) {
      const double wgt = (mm == 0 || mm == m.mz / 2) ? 1.0 : 2.0;
      const long q = ((long)mm * (m.z0 + j)) % m.mz;
      W[(size_t)mm * L.nz + j] = (float)(wgt * std::cos(2.0 * pi * q / m.mz) * scale);
    }
  unsigned long long* u_d = nullptr;
  float* W_d = nullptr;
  auto cleanup = [&]() {
    dev_free(u_d);
    dev_free(W_d);
  };
#define GEN_CUDA(call)                \
  do {                                \
    cudaError_t e_ = (call);          \
    if (e_ != cudaSuccess) {          \
      int rc_ = cuda_fail(e_, #call); \
      cleanup();                      \
      return rc_;                     \
    }                                 \
  } while (0)
  GEN_CUDA(dev_alloc(&u_d, u.size() * sizeof(unsigned long long)));
  GEN_CUDA(dev_alloc(&W_d, W.size() * sizeof(float)));
  GEN_CUDA(cudaMemcpy(u_d, u.data(), u.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice));
  GEN_CUDA(cudaMemcpy(W_d, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice));
  GEN_CUDA(dev_alloc(&p.table, L.table_bytes));
  GEN_CUDA(cudaMemsetAsync(p.table, 0, L.table_bytes, s));
  const size_t smem = sizeof(float) * ((size_t)M * L.nz + (size_t)M * 32);
  if (smem > 227 * 1024) {
    cleanup();
    return fail(PAT_ERR_UNSUPPORTED, "k-space generator: (mz/2 + 1) * (nz + 32) floats exceed shared memory");
  }
  GEN_CUDA(cudaFuncSetAttribute((const void*)k_kspace, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  if (npos > 0) {  // a frequency shard may hold no rows
    k_kspace<<<(unsigned)((npos + 31) / 32), 256, smem, s>>>(L.px, L.py, m.mz, L.nz, L.nt, L.nzg,
                                                              L.zg, L.real ? 0 : 1, u_d, W_d,
                                                              p.table, npos);
    GEN_CUDA(cudaGetLastError());
  }
  GEN_CUDA(cudaStreamSynchronize(s));
  cleanup();
  p.table_max_abs = 0;
  p.table_max_imag = 0;
  return PAT_OK;
#undef GEN_CUDA
}

}  // namespace pat

extern "C" int pat_fold_blocks(int P, int radial, int64_t* nrb, int64_t* nch, int32_t* rb_rep,
                               int32_t* rb_chunk, int32_t* row_rep, int32_t* rep_row) {
  using namespace pat;
  try {
    if (!nrb || !nch) return fail(PAT_ERR_ARG, "nrb or nch is NULL");
    if (P < 2 || P > 65536 || (P & 1)) return fail(PAT_ERR_ARG, "P must be even, in [2, 65536]");
    std::vector<int> members, rep, slot;
    fold_enumerate(P, members, rep, slot);
    const int64_t U = (int64_t)members.size() / 4;
    FoldBlocks fb;
    fold_blocks(P, members, U, radial != 0, fb);
    *nrb = fb.nrb;
    *nch = fb.nch;
    if (rb_rep) std::copy(fb.rb_rep.begin(), fb.rb_rep.end(), rb_rep);
    if (rb_chunk) std::copy(fb.rb_chunk.begin(), fb.rb_chunk.end(), rb_chunk);
    if (row_rep) std::copy(fb.row_rep.begin(), fb.row_rep.end(), row_rep);
    if (rep_row) std::copy(fb.rep_row.begin(), fb.rep_row.end(), rep_row);
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_OOM, "host allocation failed");
  }
}
