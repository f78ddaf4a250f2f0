/*
 * CPU oracle for the planar photoacoustic forward operator H, its adjoint H*,
 * and the k-space wave solve that produces the impulse-response library.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this code; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no source, header, table or helper with
 * the CUDA path.
 *
 * Everything is IEEE double precision and written as the plain definitions of
 * the paper (Küçükkömürcü, Labouesse, Allain, Chaigne, "A depth-dependent,
 * transverse shift-invariant operator for fast iterative 3D photoacoustic
 * tomography in planar geometry"):
 *   - Eq. 7 / Eq. 8   forward operator d = H rho (sum over depth of transverse
 *                     2D convolutions with the depth-indexed kernels h_z)
 *   - Eq. 9-11        adjoint H* under the Euclidean inner products (sum over
 *                     time of transverse 2D correlations)
 *   - Sec. 2.3 end    FFT realisation with zero-padding and cropping
 *   - Eq. 1-2         homogeneous wave equation, p(r,0)=p0, dp/dt(r,0)=0,
 *                     solved with an exact k-space propagator on a periodic grid
 *   - Sec. 3.2        one point-source solve, recorded on every depth plane,
 *                     gives the whole library (reciprocity)
 *
 * Array conventions (row-major, x fastest):
 *   rho  [nz][ny][nx]          object, depth plane j sits at z = (z0 + j) dz
 *   d    [nt][ny][nx]          sensor data on the plane z = 0, t_n = n dt
 *   h    [nz][nt][py][px]      spatial kernels; displacement (ux,uy) is stored at
 *                              index (ux mod px, uy mod py) ("wrapped origin")
 *   Hf   [nz][nt][py][px]      full-plane spectra of h, complex (re,im) pairs,
 *                              unnormalised forward DFT exp(-2 pi i k n / P)
 * Complex arrays are interleaved (re, im) doubles.
 *
 * Return codes: 0 on success, -1 on bad arguments (sizes not positive, a
 * padded size that is not a power of two or is smaller than 2n-1).
 */
#ifndef PAT_ORACLE_H
#define PAT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Number of worker threads (0 = all hardware threads). */
void orc_set_threads(int n);
int orc_get_threads(void);

/* 1D DFTs of a contiguous complex vector of length n.
 * orc_fft1d: own radix-2 FFT, in place, n a power of two.
 * orc_dft1d: the O(n^2) definition, out-of-place, any n.
 * inverse = 0 uses exp(-2 pi i k m / n); inverse = 1 uses exp(+...). Neither
 * normalises. */
int orc_fft1d(double* a, long n, int inverse);
int orc_dft1d(const double* in, double* out, long n, int inverse);

/* In-place 2D / 3D FFT of a contiguous complex array [py][px] / [mz][py][px]. */
int orc_fft2d(double* a, long py, long px, int inverse);
int orc_fft3d(double* a, long mz, long py, long px, int inverse);

/* Eq. 7, written out: d[t][s] = sum_j sum_r h[j][t][(s - r) mod P] rho[j][r]. */
int orc_forward_spatial(const double* h, const double* rho, double* d,
                        long nx, long ny, long nz, long nt, long px, long py);
/* Eq. 11, written out: rho[j][r] = sum_t sum_s h[j][t][(s - r) mod P] d[t][s]. */
int orc_adjoint_spatial(const double* h, const double* d, double* rho,
                        long nx, long ny, long nz, long nt, long px, long py);

/* Hf[j][t] = DFT2(h[j][t]). */
int orc_table_spectrum(const double* h, double* Hf, long nz, long nt, long px, long py);

/* FFT realisation of Eq. 7 (zero-pad to P, DFT, multiply-accumulate over depth
 * for every time sample, inverse DFT, crop to the first n x n samples). */
int orc_forward_fft(const double* Hf, const double* rho, double* d,
                    long nx, long ny, long nz, long nt, long px, long py);
/* FFT realisation of Eq. 11 (the exact transpose of orc_forward_fft). */
int orc_adjoint_fft(const double* Hf, const double* d, double* rho,
                    long nx, long ny, long nz, long nt, long px, long py);

/* Homogeneous, lossless medium and the sampling steps. */
typedef struct {
  double c;   /* sound speed [m/s] */
  double dx;  /* grid steps [m] */
  double dy;
  double dz;
  double dt;  /* time step [s] */
} orc_medium;

/* Eq. 1-2 on a periodic px x py x mz grid with the exact k-space propagator.
 * p0 [mz][py][px]; records the planes listed in planes[] at t_n = n dt,
 * n = 0..nt-1, into rec[nplanes][nt][py][px].
 * closed_form = 1: p^(k, t_n) = cos(c |k| t_n) p0^(k).
 * closed_form = 0: time stepping p^{n+1} = 2 cos(c|k|dt) p^n - p^{n-1},
 *                  p^1 = cos(c|k|dt) p^0 (from dp/dt = 0 at t = 0). */
int orc_kspace_solve(const double* p0, long px, long py, long mz, orc_medium m,
                     long nt, int closed_form, const long* planes, long nplanes,
                     double* rec);

/* The impulse-response library from ONE solve (Sec. 3.2): a unit point source
 * at (x, y, z) = (0, 0, src_plane); h[j][t] is the field recorded on plane
 * (src_plane + sign * (z0 + j)) mod mz, sign = +1 or -1. With src_plane = 0 and
 * sign = +1 the library is indexed like the object depths z = (z0 + j) dz; the
 * paper's variant puts the source at the bottom plane and records upward
 * (sign = -1). Uses the time-stepping solve. */
int orc_table_kspace_solve(long px, long py, long mz, orc_medium m, long nt,
                           long nz, long z0, long src_plane, int sign, double* h);

/* Spectrum of the same library straight from the closed form of the solve:
 * Hf[j][t][ky][kx] = (1/mz) sum_m cos(c t |k|) cos(2 pi m (z0 + j) / mz),
 * |k|^2 = kx^2 + ky^2 + kz_m^2, for the listed time indices t_idx[] and depth
 * indices z_idx[] (j in [0, nz)). Output [n_z][n_t][py][px] complex. */
int orc_table_kspace_closed(long px, long py, long mz, orc_medium m, long z0,
                            const long* t_idx, long n_t, const long* z_idx, long n_z,
                            double* Hf);

#ifdef __cplusplus
}
#endif
#endif
