// CPU oracle: plain FP64 restatement of the paper's operator and wave solve.
// TEST INFRASTRUCTURE ONLY (see pat_oracle.h). Portable C++17, no intrinsics.
#include "pat_oracle.h"

#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

typedef std::complex<double> cplx;

static int g_threads = 0;

extern "C" void orc_set_threads(int n) { g_threads = n < 0 ? 0 : n; }

extern "C" int orc_get_threads(void) {
  if (g_threads > 0) return g_threads;
  unsigned hc = std::thread::hardware_concurrency();
  return hc == 0 ? 1 : (int)hc;
}

// Runs f(i) for i in [0, n) on the worker threads (dynamic assignment).
template <class F>
static void parallel_for(long n, F f) {
  int nthr = orc_get_threads();
  if (nthr > n) nthr = (int)n;
  if (nthr <= 1) {
    for (long i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<long> next(0);
  std::vector<std::thread> pool;
  pool.reserve(nthr);
  for (int k = 0; k < nthr; ++k)
    pool.emplace_back([&]() {
      for (;;) {
        long i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& th : pool) th.join();
}

static bool is_pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }
// Transverse transform lengths: powers of two, or three times a power of two.
static bool fft_len_ok(long n) { return is_pow2(n) || (n > 0 && n % 3 == 0 && is_pow2(n / 3)); }

static const double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// FFT: iterative radix-2 Cooley-Tukey (bit-reversal permutation followed by
// log2(n) butterfly passes) for powers of two; for other lengths the DFT of
// its definition, sum_m a[m] w^(k m). Twiddles w_n^k = exp(-+2 pi i k / n)
// come from std::cos / std::sin in double precision, one table per length.
// ---------------------------------------------------------------------------
struct Twiddle {
  long n = 0;
  std::vector<cplx> w;  // w[k] = exp(-2 pi i k / n), k < n
  explicit Twiddle(long n_) : n(n_), w(n_ > 0 ? n_ : 1) {
    for (long k = 0; k < n; ++k) {
      double a = -2.0 * kPi * (double)k / (double)n;
      w[k] = cplx(std::cos(a), std::sin(a));
    }
  }
};

static void dft_inplace(cplx* a, const Twiddle& tw, int inverse) {
  const long n = tw.n;
  std::vector<cplx> out(n);
  for (long k = 0; k < n; ++k) {
    cplx acc(0.0, 0.0);
    for (long m = 0; m < n; ++m) {
      cplx w = tw.w[(k * m) % n];
      if (inverse) w = std::conj(w);
      acc += a[m] * w;
    }
    out[k] = acc;
  }
  for (long k = 0; k < n; ++k) a[k] = out[k];
}

static void fft_inplace(cplx* a, const Twiddle& tw, int inverse) {
  const long n = tw.n;
  if (!is_pow2(n)) {
    dft_inplace(a, tw, inverse);
    return;
  }
  for (long i = 1, j = 0; i < n; ++i) {
    long bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (long len = 2; len <= n; len <<= 1) {
    const long half = len / 2, step = n / len;
    for (long i = 0; i < n; i += len) {
      for (long k = 0; k < half; ++k) {
        cplx w = tw.w[k * step];
        if (inverse) w = std::conj(w);
        cplx u = a[i + k];
        cplx v = a[i + k + half] * w;
        a[i + k] = u + v;
        a[i + k + half] = u - v;
      }
    }
  }
}

// 2D transform of one contiguous [py][px] plane: rows, then columns.
static void fft2_plane(cplx* a, long py, long px, const Twiddle& twx,
                       const Twiddle& twy, int inverse, std::vector<cplx>& col) {
  for (long y = 0; y < py; ++y) fft_inplace(a + y * px, twx, inverse);
  col.resize(py);
  for (long x = 0; x < px; ++x) {
    for (long y = 0; y < py; ++y) col[y] = a[y * px + x];
    fft_inplace(col.data(), twy, inverse);
    for (long y = 0; y < py; ++y) a[y * px + x] = col[y];
  }
}

extern "C" int orc_fft1d(double* a, long n, int inverse) {
  if (!fft_len_ok(n) || a == nullptr) return -1;
  Twiddle tw(n);
  fft_inplace(reinterpret_cast<cplx*>(a), tw, inverse);
  return 0;
}

extern "C" int orc_dft1d(const double* in, double* out, long n, int inverse) {
  if (n <= 0 || in == nullptr || out == nullptr) return -1;
  const cplx* x = reinterpret_cast<const cplx*>(in);
  cplx* y = reinterpret_cast<cplx*>(out);
  const double sgn = inverse ? 1.0 : -1.0;
  for (long k = 0; k < n; ++k) {
    cplx acc(0.0, 0.0);
    for (long m = 0; m < n; ++m) {
      // reduce k*m mod n before the angle so large products stay exact
      double a = sgn * 2.0 * kPi * (double)((k * m) % n) / (double)n;
      acc += x[m] * cplx(std::cos(a), std::sin(a));
    }
    y[k] = acc;
  }
  return 0;
}

extern "C" int orc_fft2d(double* a, long py, long px, int inverse) {
  if (!fft_len_ok(px) || !fft_len_ok(py) || a == nullptr) return -1;
  Twiddle twx(px), twy(py);
  std::vector<cplx> col;
  fft2_plane(reinterpret_cast<cplx*>(a), py, px, twx, twy, inverse, col);
  return 0;
}

extern "C" int orc_fft3d(double* a, long mz, long py, long px, int inverse) {
  if (!fft_len_ok(px) || !fft_len_ok(py) || !is_pow2(mz) || a == nullptr) return -1;
  cplx* c = reinterpret_cast<cplx*>(a);
  Twiddle twx(px), twy(py), twz(mz);
  parallel_for(mz, [&](long z) {
    std::vector<cplx> col;
    fft2_plane(c + z * py * px, py, px, twx, twy, inverse, col);
  });
  const long plane = py * px;
  parallel_for(plane, [&](long i) {
    std::vector<cplx> v(mz);
    for (long z = 0; z < mz; ++z) v[z] = c[z * plane + i];
    fft_inplace(v.data(), twz, inverse);
    for (long z = 0; z < mz; ++z) c[z * plane + i] = v[z];
  });
  return 0;
}

// ---------------------------------------------------------------------------
// Operator checks shared by the operator entry points.
// ---------------------------------------------------------------------------
static bool geom_ok(long nx, long ny, long nz, long nt, long px, long py) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || nt <= 0) return false;
  if (!fft_len_ok(px) || !fft_len_ok(py)) return false;
  // linear (not circular) convolution needs P >= 2n - 1
  if (px < 2 * nx - 1 || py < 2 * ny - 1) return false;
  return true;
}

static inline long wrap(long v, long p) {
  long r = v % p;
  return r < 0 ? r + p : r;
}

// Eq. 7: d(r_perp, t) = sum over depths of h_z(., t) convolved with rho(., z).
extern "C" int orc_forward_spatial(const double* h, const double* rho, double* d,
                                   long nx, long ny, long nz, long nt, long px,
                                   long py) {
  if (!geom_ok(nx, ny, nz, nt, px, py) || !h || !rho || !d) return -1;
  const long plane = px * py;
  parallel_for(nt, [&](long t) {
    for (long sy = 0; sy < ny; ++sy)
      for (long sx = 0; sx < nx; ++sx) {
        double acc = 0.0;
        for (long j = 0; j < nz; ++j) {
          const double* hk = h + (j * nt + t) * plane;
          const double* rj = rho + j * ny * nx;
          for (long ry = 0; ry < ny; ++ry)
            for (long rx = 0; rx < nx; ++rx)
              acc += hk[wrap(sy - ry, py) * px + wrap(sx - rx, px)] * rj[ry * nx + rx];
        }
        d[(t * ny + sy) * nx + sx] = acc;
      }
  });
  return 0;
}

// Eq. 11: (H* d)(r_perp, z) = sum over time of h_z(., t) correlated with d(., t).
extern "C" int orc_adjoint_spatial(const double* h, const double* d, double* rho,
                                   long nx, long ny, long nz, long nt, long px,
                                   long py) {
  if (!geom_ok(nx, ny, nz, nt, px, py) || !h || !rho || !d) return -1;
  const long plane = px * py;
  parallel_for(nz, [&](long j) {
    for (long ry = 0; ry < ny; ++ry)
      for (long rx = 0; rx < nx; ++rx) {
        double acc = 0.0;
        for (long t = 0; t < nt; ++t) {
          const double* hk = h + (j * nt + t) * plane;
          const double* dt_ = d + t * ny * nx;
          for (long sy = 0; sy < ny; ++sy)
            for (long sx = 0; sx < nx; ++sx)
              acc += hk[wrap(sy - ry, py) * px + wrap(sx - rx, px)] * dt_[sy * nx + sx];
        }
        rho[(j * ny + ry) * nx + rx] = acc;
      }
  });
  return 0;
}

extern "C" int orc_table_spectrum(const double* h, double* Hf, long nz, long nt,
                                  long px, long py) {
  if (nz <= 0 || nt <= 0 || !fft_len_ok(px) || !fft_len_ok(py) || !h || !Hf) return -1;
  const long plane = px * py;
  Twiddle twx(px), twy(py);
  cplx* out = reinterpret_cast<cplx*>(Hf);
  parallel_for(nz * nt, [&](long s) {
    std::vector<cplx> col;
    cplx* a = out + s * plane;
    for (long i = 0; i < plane; ++i) a[i] = cplx(h[s * plane + i], 0.0);
    fft2_plane(a, py, px, twx, twy, 0, col);
  });
  return 0;
}

// Zero-padding of an [ny][nx] real slice into a [py][px] complex plane at the
// top-left corner (indices [0, ny) x [0, nx)), followed by a forward 2D DFT.
static void pad_fft(const double* src, long nx, long ny, long px, long py,
                    const Twiddle& twx, const Twiddle& twy, cplx* dst,
                    std::vector<cplx>& col) {
  for (long i = 0; i < px * py; ++i) dst[i] = cplx(0.0, 0.0);
  for (long y = 0; y < ny; ++y)
    for (long x = 0; x < nx; ++x) dst[y * px + x] = cplx(src[y * nx + x], 0.0);
  fft2_plane(dst, py, px, twx, twy, 0, col);
}

// Inverse 2D DFT (with the 1/(px py) factor) and crop back to [ny][nx]; the
// real part is kept (the imaginary part is rounding noise for real data).
static void ifft_crop(cplx* a, long nx, long ny, long px, long py,
                      const Twiddle& twx, const Twiddle& twy, double* dst,
                      std::vector<cplx>& col) {
  fft2_plane(a, py, px, twx, twy, 1, col);
  const double s = 1.0 / (double)(px * py);
  for (long y = 0; y < ny; ++y)
    for (long x = 0; x < nx; ++x) dst[y * nx + x] = a[y * px + x].real() * s;
}

// Eq. 7 evaluated in the Fourier domain: X_j = F(pad rho_j);
// Y_t = sum_j Hf[j][t] X_j; d_t = crop(F^-1 Y_t).
extern "C" int orc_forward_fft(const double* Hf, const double* rho, double* d,
                               long nx, long ny, long nz, long nt, long px,
                               long py) {
  if (!geom_ok(nx, ny, nz, nt, px, py) || !Hf || !rho || !d) return -1;
  const long plane = px * py;
  const cplx* H = reinterpret_cast<const cplx*>(Hf);
  Twiddle twx(px), twy(py);
  std::vector<cplx> X((size_t)(nz * plane));
  parallel_for(nz, [&](long j) {
    std::vector<cplx> col;
    pad_fft(rho + j * ny * nx, nx, ny, px, py, twx, twy, X.data() + j * plane, col);
  });
  parallel_for(nt, [&](long t) {
    std::vector<cplx> Y((size_t)plane, cplx(0.0, 0.0)), col;
    for (long j = 0; j < nz; ++j) {
      const cplx* Hk = H + (j * nt + t) * plane;
      const cplx* Xj = X.data() + j * plane;
      for (long i = 0; i < plane; ++i) Y[i] += Hk[i] * Xj[i];
    }
    ifft_crop(Y.data(), nx, ny, px, py, twx, twy, d + t * ny * nx, col);
  });
  return 0;
}

// Eq. 11 in the Fourier domain: D_t = F(pad d_t);
// Z_j = sum_t conj(Hf[j][t]) D_t; rho_j = crop(F^-1 Z_j).
extern "C" int orc_adjoint_fft(const double* Hf, const double* d, double* rho,
                               long nx, long ny, long nz, long nt, long px,
                               long py) {
  if (!geom_ok(nx, ny, nz, nt, px, py) || !Hf || !rho || !d) return -1;
  const long plane = px * py;
  const cplx* H = reinterpret_cast<const cplx*>(Hf);
  Twiddle twx(px), twy(py);
  std::vector<cplx> D((size_t)(nt * plane));
  parallel_for(nt, [&](long t) {
    std::vector<cplx> col;
    pad_fft(d + t * ny * nx, nx, ny, px, py, twx, twy, D.data() + t * plane, col);
  });
  parallel_for(nz, [&](long j) {
    std::vector<cplx> Z((size_t)plane, cplx(0.0, 0.0)), col;
    for (long t = 0; t < nt; ++t) {
      const cplx* Hk = H + (j * nt + t) * plane;
      const cplx* Dt = D.data() + t * plane;
      for (long i = 0; i < plane; ++i) Z[i] += std::conj(Hk[i]) * Dt[i];
    }
    ifft_crop(Z.data(), nx, ny, px, py, twx, twy, rho + j * ny * nx, col);
  });
  return 0;
}

// ---------------------------------------------------------------------------
// k-space solve of Eq. 1-2 on a periodic grid.
// ---------------------------------------------------------------------------

// Angular wavenumber of DFT index m on a grid of n points with spacing step:
// 2 pi m_s / (n step) with the signed index m_s in [-n/2, n/2).
static inline double wavenumber(long m, long n, double step) {
  long ms = (m < n / 2) ? m : m - n;
  return 2.0 * kPi * (double)ms / ((double)n * step);
}

extern "C" int orc_kspace_solve(const double* p0, long px, long py, long mz,
                                orc_medium med, long nt, int closed_form,
                                const long* planes, long nplanes, double* rec) {
  if (!fft_len_ok(px) || !fft_len_ok(py) || !is_pow2(mz) || nt <= 0 || nplanes <= 0 ||
      !p0 || !planes || !rec)
    return -1;
  for (long p = 0; p < nplanes; ++p)
    if (planes[p] < 0 || planes[p] >= mz) return -1;
  const long plane = px * py, vol = plane * mz;
  std::vector<cplx> P0((size_t)vol);
  for (long i = 0; i < vol; ++i) P0[i] = cplx(p0[i], 0.0);
  orc_fft3d(reinterpret_cast<double*>(P0.data()), mz, py, px, 0);

  // |k| for every mode.
  std::vector<double> kmag((size_t)vol);
  for (long z = 0; z < mz; ++z)
    for (long y = 0; y < py; ++y)
      for (long x = 0; x < px; ++x) {
        double kx = wavenumber(x, px, med.dx), ky = wavenumber(y, py, med.dy),
               kz = wavenumber(z, mz, med.dz);
        kmag[(z * py + y) * px + x] = std::sqrt(kx * kx + ky * ky + kz * kz);
      }

  std::vector<cplx> prev, cur, nxt((size_t)vol), work((size_t)vol);
  std::vector<double> c1((size_t)vol);  // cos(c |k| dt)
  for (long i = 0; i < vol; ++i) c1[i] = std::cos(med.c * kmag[i] * med.dt);
  if (!closed_form) {
    prev = P0;  // step 0: p^0 = p0^
    cur.resize((size_t)vol);
    for (long i = 0; i < vol; ++i) cur[i] = c1[i] * P0[i];  // step 1
  }
  const double s = 1.0 / (double)vol;
  for (long n = 0; n < nt; ++n) {
    if (closed_form) {
      const double tn = (double)n * med.dt;
      for (long i = 0; i < vol; ++i) work[i] = std::cos(med.c * kmag[i] * tn) * P0[i];
    } else if (n == 0) {
      work = prev;
    } else if (n == 1) {
      work = cur;
    } else {
      // p^{n} = 2 cos(c|k|dt) p^{n-1} - p^{n-2}
      for (long i = 0; i < vol; ++i) nxt[i] = 2.0 * c1[i] * cur[i] - prev[i];
      prev.swap(cur);
      cur.swap(nxt);
      work = cur;
    }
    orc_fft3d(reinterpret_cast<double*>(work.data()), mz, py, px, 1);
    for (long p = 0; p < nplanes; ++p) {
      const cplx* src = work.data() + planes[p] * plane;
      double* dst = rec + (p * nt + n) * plane;
      for (long i = 0; i < plane; ++i) dst[i] = src[i].real() * s;
    }
  }
  return 0;
}

extern "C" int orc_table_kspace_solve(long px, long py, long mz, orc_medium med,
                                      long nt, long nz, long z0, long src_plane,
                                      int sign, double* h) {
  if (nz <= 0 || nt <= 0 || !is_pow2(mz) || !h || (sign != 1 && sign != -1) ||
      src_plane < 0 || src_plane >= mz)
    return -1;
  const long plane = px * py;
  std::vector<double> p0((size_t)(plane * mz), 0.0);
  p0[(size_t)(src_plane * plane)] = 1.0;  // unit-amplitude point absorber
  std::vector<long> planes((size_t)nz);
  for (long j = 0; j < nz; ++j) planes[j] = wrap(src_plane + sign * (z0 + j), mz);
  return orc_kspace_solve(p0.data(), px, py, mz, med, nt, 0, planes.data(), nz, h);
}

extern "C" int orc_table_kspace_closed(long px, long py, long mz, orc_medium med,
                                       long z0, const long* t_idx, long n_t,
                                       const long* z_idx, long n_z, double* Hf) {
  if (!fft_len_ok(px) || !fft_len_ok(py) || !is_pow2(mz) || n_t <= 0 || n_z <= 0 ||
      !t_idx || !z_idx || !Hf)
    return -1;
  const long plane = px * py;
  // cz[jj][m] = cos(2 pi m (z0 + j) / mz) = cos(kz_m z_j)
  std::vector<double> cz((size_t)(n_z * mz));
  for (long jj = 0; jj < n_z; ++jj)
    for (long m = 0; m < mz; ++m) {
      long q = (m * (z0 + z_idx[jj])) % mz;  // exact phase index
      cz[jj * mz + m] = std::cos(2.0 * kPi * (double)q / (double)mz);
    }
  cplx* out = reinterpret_cast<cplx*>(Hf);
  parallel_for(n_t * py, [&](long task) {
    const long tt = task / py, y = task % py;
    const double tn = (double)t_idx[tt] * med.dt;
    const double ky = wavenumber(y, py, med.dy);
    std::vector<double> ct((size_t)mz);
    for (long x = 0; x < px; ++x) {
      const double kx = wavenumber(x, px, med.dx);
      for (long m = 0; m < mz; ++m) {
        const double kz = wavenumber(m, mz, med.dz);
        ct[m] = std::cos(med.c * tn * std::sqrt(kx * kx + ky * ky + kz * kz));
      }
      for (long jj = 0; jj < n_z; ++jj) {
        double acc = 0.0;
        for (long m = 0; m < mz; ++m) acc += ct[m] * cz[jj * mz + m];
        out[(jj * n_t + tt) * plane + y * px + x] = cplx(acc / (double)mz, 0.0);
      }
    }
  });
  return 0;
}
