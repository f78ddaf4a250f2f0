/*
 * pat.h -- C ABI of the GB300 photoacoustic operator library (libpat.so).
 *
 * The library applies the planar-geometry photoacoustic forward operator H of
 * Küçükkömürcü, Labouesse, Allain & Chaigne ("A depth-dependent, transverse
 * shift-invariant operator for fast iterative 3D photoacoustic tomography in
 * planar geometry"), its discrete adjoint H*, and FISTA on top of them, with
 * hand-written CUDA kernels for sm_103a.
 *
 *   Eq. 7-8   d(r, t)   = sum_z  h_z(., t) (*) rho(., z)        (forward)
 *   Eq. 9-11  H*d(r, z) = sum_t  h_z(., t) (x) d(., t)          (adjoint: correlation)
 *   Eq. 12-15 FISTA for 1/2 ||H rho - d||^2 + lambda ||rho||_1 + indicator(rho >= 0)
 *
 * Both operators run as three stages (Sec. 3.2, Eq. 16): zero-padded 2D real
 * FFTs of every slice, a per-frequency contraction with the stored spectra of
 * the impulse-response library, and cropped 2D inverse FFTs.
 *
 * ---------------------------------------------------------------------------
 * Conventions (every entry point)
 *   Arrays are dense, row-major, x fastest:
 *     object rho [batch][nz][ny][nx],  data d [batch][nt][my][mx],
 *   where (my, mx) = (ny, nx) unless pat_plan_set_sampling put the data on a
 *   coarser scan grid. Below, "[ny][nx]" of data means [my][mx].
 *   Element type: float for single-precision plans, double for plans created
 *   with PAT_FLAG_FP64 ("real_t" below).
 *   Pointers may be device memory (the normal case; the call is asynchronous on
 *   `stream`) or host memory (pageable or pinned): host arrays are copied
 *   through plan-owned device staging buffers and the call returns after the
 *   result is back in host memory.
 *   The caller owns every array it passes; the library keeps no pointer to
 *   them after a call returns. A plan owns its table copy (the resident
 *   spectral layout, built at creation). Its workspace (every per-call buffer)
 *   is either allocated by the plan (pat_plan_create*) or caller-owned device
 *   memory sized by pat_workspace_size (pat_plan_create*_with_workspace).
 *   `stream` is a cudaStream_t (0 = legacy default stream).
 *   Calls on one plan must not overlap (one plan = one stream of work); plans
 *   are independent of each other.
 * Errors
 *   Every int-returning function returns PAT_OK (0) or a negative pat_status.
 *   No C++ exception crosses the ABI. On an argument error nothing is launched
 *   and outputs are untouched. pat_last_error() gives a message for the last
 *   failure on the calling thread.
 * ---------------------------------------------------------------------------
 */
#ifndef PAT_H
#define PAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pat_plan pat_plan;       /* opaque */
typedef struct CUstream_st* pat_stream; /* the same handle as cudaStream_t */

typedef enum {
  PAT_OK = 0,
  PAT_ERR_ARG = -1,         /* invalid argument (size, pointer, format, batch)  */
  PAT_ERR_OOM = -2,         /* device or host allocation failed                  */
  PAT_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed       */
  PAT_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up                */
  PAT_ERR_UNSUPPORTED = -5  /* valid request this build does not implement       */
} pat_status;

enum {
  PAT_FLAG_FP64 = 1,          /* table, workspace and arrays in double precision */
  PAT_FLAG_FORCE_COMPLEX = 2, /* keep the complex table even when it is real     */
  PAT_FLAG_NO_FOLD = 8,       /* keep one table row per bin even when the spectra have
                                 the D4 symmetry of radially symmetric kernels */
  PAT_FLAG_NO_RADIAL = 16,    /* folded plans: keep one stored row per D4
                                 representative even when representatives of equal
                                 kx^2 + ky^2 have equal spectra */
  PAT_FLAG_BF16_SPLIT = 4     /* also build the split-BF16 tensor-core tables: calls
                                 with batch >= 2 contract 16 volumes per table pass on
                                 tcgen05 (BF16 hi/lo operands, FP32 accumulation).
                                 Needs a real table, nz = 128, nt in {128, 256, 384, 512},
                                 single precision; else pat_plan_create fails with
                                 PAT_ERR_UNSUPPORTED. Folded plans keep one tile set
                                 per representative and contract its bins together. */
};

/* Grid of one plan.
 *   nx, ny   transverse grid of rho and d (Sec. 2.2, G_xy)
 *   nz       depth planes of rho (G_z);  nt  time samples of d (T)
 *   px, py   padded transverse grid for linear convolution (Sec. 2.3, end):
 *            2^k or 3 * 2^k (16, 24, 32, 48, ..., 768, 1024), px >= 2 nx - 1,
 *            py >= 2 ny - 1; other lengths return PAT_ERR_UNSUPPORTED
 *   max_batch  largest `batch` any call on this plan may pass (sizes workspace)
 *   flags    PAT_FLAG_* */
typedef struct {
  int32_t nx, ny, nz, nt;
  int32_t px, py;
  int32_t max_batch;
  int32_t flags;
} pat_geometry;

/* Layout of the impulse-response library handed to pat_plan_create.
 * SPATIAL: h[nz][nt][py][px] real; the kernel value for transverse
 *   displacement (ux, uy) sits at [uy mod py][ux mod px] ("wrapped origin");
 *   constant discretisation factors are already folded in (Sec. 2.2).
 * SPECTRAL: Hh[nz][nt][py][px/2 + 1] complex (re, im interleaved), the
 *   non-negative-kx half of the unnormalised 2D DFT exp(-2 pi i k.n / P) of h. */
typedef enum {
  PAT_TABLE_SPATIAL_F64 = 0,
  PAT_TABLE_SPATIAL_F32 = 1,
  PAT_TABLE_SPECTRAL_C128 = 2,
  PAT_TABLE_SPECTRAL_C64 = 3
} pat_table_format;

/* Homogeneous lossless medium for a library generated on the device from the
 * exact k-space solution of Eq. 1-2 on a periodic px x py x mz grid (one
 * unit point source, recorded on the planes z = (z0 + j) dz, Sec. 3.2):
 *   Hh[j][t](kx, ky) = (1/mz) sum_m cos(c t dt |k|) cos(2 pi m (z0 + j) / mz),
 *   |k|^2 = kx^2 + ky^2 + (2 pi m_s / (mz dz))^2, m_s the signed index of m. */
typedef struct {
  double c;          /* sound speed [m/s] */
  double dx, dy, dz; /* voxel steps [m] */
  double dt;         /* sampling step [s]; t_n = n dt, n = 0..nt-1 */
  int32_t mz;        /* depth period of the solve: power of two > z0 + nz */
  int32_t z0;        /* index of the first object plane (>= 0) */
} pat_medium;

/* Information about a plan (filled by pat_plan_info). */
typedef struct {
  int32_t real_table;      /* 1: the stored spectra are real (even kernels) */
  int32_t fp64;            /* 1: double-precision plan */
  int64_t bins;            /* stored frequency bins K = (px/2 + 1) py */
  int64_t bins_padded;     /* K rounded up to a multiple of 32 (row stride of stage ii) */
  int64_t table_bytes;     /* device bytes of the resident table */
  int64_t workspace_bytes; /* device bytes of the plan's workspace */
  double table_max_abs;    /* max |Hh| seen while building the table */
  double table_max_imag;   /* max |Im Hh| seen while building the table */
  int64_t tensor_table_bytes; /* device bytes of the split-BF16 tables (0 if not built) */
  int32_t tensor_min_batch;   /* batches >= this use the tensor-core contraction (0: never) */
  int32_t folded;             /* 1: one table row per D4 representative {|kx|, |ky|} */
  int64_t table_rows;         /* frequency rows: representatives if folded, else bins */
  int32_t workspace_external; /* 1: the workspace is caller-owned memory */
  int32_t radial;             /* 1: folded, and representatives with equal kx^2 + ky^2
                                 share one stored row (see pat_fold_blocks) */
  int64_t stored_rows;        /* rows held in device memory (padded to 32):
                                 table_bytes = stored_rows * nt * nz * element size */
} pat_plan_info_t;

/* FISTA settings (Eq. 12-14; Beck & Teboulle's constant-step scheme).
 *   iters       iterations (>= 0)
 *   lambda      l1 weight of Eq. 14 (>= 0); lambda = 0 gives non-negative least squares
 *   L           Lipschitz constant ||H*H|| used as step 1/L; L <= 0 asks the
 *               solver to estimate it with pat_power_norm (power_iters steps
 *               from a fixed-seed start vector) and multiply by 1.01
 *   power_iters steps of that estimate (ignored when L > 0)
 *   warm_start  1: start from the x passed in; 0: start from zero */
typedef struct {
  int32_t iters;
  int32_t power_iters;
  int32_t warm_start;
  int32_t reserved;
  double lambda;
  double L;
} pat_fista_params;

/* What pat_fista_solve reports (written after the solve has finished). */
typedef struct {
  double L;             /* step-size constant actually used */
  double resid2_first;  /* ||H y_1 - d||^2 of the first gradient step (batch sum) */
  double resid2_last;   /* ||H y_k - d||^2 of the last gradient step (batch sum) */
  int32_t iters;        /* iterations run */
  int32_t kernels_per_iter; /* kernel launches of one iteration (graph kernel nodes) */
} pat_fista_report;

/* --- plans ------------------------------------------------------------------ */

/* Builds a plan: validates the grid, allocates the device table and workspace,
 * and converts `table` (host or device memory, layout `fmt`) into the plan's
 * resident spectral layout. The spectra are scaled by 1/(px py) once here so
 * the inverse FFTs need no normalisation. When every |Im Hh| <= 1e-6 max |Hh|
 * (kernels even under (x, y) -> (-x, -y), e.g. the radially symmetric
 * kernels of Eq. 5) and PAT_FLAG_FORCE_COMPLEX is not set, the imaginary part
 * is dropped and the real-spectrum contraction is used (half the bytes).
 * A real table on a square padded grid whose spectra also agree (to 1e-6 of
 * max |Hh|) under ky -> -ky and kx <-> ky -- kernels with the radial symmetry
 * of Eq. 5 -- is stored once per representative {|kx|, |ky|} ("folded", ~4x
 * fewer bytes; the bins of a representative share its row) unless
 * PAT_FLAG_NO_FOLD is set. A folded table whose representatives of equal
 * kx^2 + ky^2 also agree (to the same 1e-6) -- spectra that depend on |k| only,
 * as Eq. 5's do for a homogeneous medium on an isotropic grid -- keeps one
 * stored row per radius group (pat_fold_blocks; ~30 % fewer bytes at P = 256)
 * unless PAT_FLAG_NO_RADIAL is set. Synchronises `stream` before returning.
 * Table source: Sec. 3.2. */
int pat_plan_create(const pat_geometry* g, const void* table, pat_table_format fmt,
                    pat_stream stream, pat_plan** out);

/* Builds a plan whose library is generated on the device from `m` (formula
 * above; Eq. 1-2 and the single-solve reciprocity construction of Sec. 3.2).
 * The generated spectra depend on kx^2 + ky^2 (and z, t) only, so with
 * dx = dy on a square padded grid the plan is folded and radial (unless
 * PAT_FLAG_NO_FOLD / PAT_FLAG_NO_RADIAL). */
int pat_plan_create_kspace(const pat_geometry* g, const pat_medium* m,
                           pat_stream stream, pat_plan** out);

/* Device bytes of the workspace of a plan for `g` (Sec. 3.2's three stages
 * need the slice spectra X / Y of Eq. 16 terms (i)-(iii) between the stages,
 * plus the FISTA state of Eq. 12-14): the spectra and FFT intermediate, three
 * object and two data buffers, FP64 reduction scratch, scalars, the slot
 * state, the FISTA history for up to 4096 iterations per solve, and the
 * host-pointer staging buffers. Returns the bytes (>= 0), or a negative
 * pat_status for an invalid geometry. No device call is made. */
int64_t pat_workspace_size(const pat_geometry* g);

/* pat_plan_create / pat_plan_create_kspace on a caller-owned workspace:
 * `workspace` is device memory of `ws_bytes` >= pat_workspace_size(g) bytes,
 * 256-byte aligned (e.g. a torch tensor's storage), which the plan uses for
 * all its per-call buffers and never frees; it must stay allocated and
 * untouched by the caller until pat_plan_destroy returns. The plan still
 * allocates its resident table (and, during creation only, the temporaries of
 * table preparation). Such a plan runs at most 4096 FISTA iterations per
 * pat_fista_solve call (PAT_ERR_ARG beyond). Errors as pat_plan_create, plus
 * PAT_ERR_ARG for a workspace that is not device memory, misaligned or too
 * small. */
int pat_plan_create_with_workspace(const pat_geometry* g, const void* table, pat_table_format fmt,
                                   void* workspace, size_t ws_bytes, pat_stream stream,
                                   pat_plan** out);
int pat_plan_create_kspace_with_workspace(const pat_geometry* g, const pat_medium* m,
                                          void* workspace, size_t ws_bytes, pat_stream stream,
                                          pat_plan** out);

/* Frees the plan's device memory (synchronises the device first); a
 * caller-owned workspace is left alone. NULL is a no-op. (Plan management:
 * no counterpart in the paper.) */
int pat_plan_destroy(pat_plan* plan);

/* Fills *info with the plan's representation of the stored library (Sec. 3.2:
 * the spectra precomputed once and kept resident; Sec. 4: their size) and its
 * sizes. No device call; PAT_ERR_ARG for a NULL plan or info. */
int pat_plan_info(const pat_plan* plan, pat_plan_info_t* info);

/* Device bytes a plan for `g` would take, before creating it (admission
 * control; the stored operator's size is the limitation Sec. 4 discusses):
 * *table_bytes for the representation of the library given by
 * real_table: 0 complex, 1 real (one row per bin), 2 real D4-folded, 3 real
 * folded with radial sharing (a k-space library with dx = dy gets 3); 2 and 3
 * need a square padded grid in single precision, else they count as 1. With
 * PAT_FLAG_BF16_SPLIT the split tensor tables (one tile set per row: per
 * representative when folded) are included. *workspace for everything else
 * (including the host-pointer staging buffers). No device call is made. */
int pat_plan_estimate(const pat_geometry* g, int real_table, int64_t* table_bytes,
                      int64_t* workspace);

/* Message of the last failure on the calling thread ("" if none). */
const char* pat_last_error(void);

/* Sets the smallest batch that uses the tensor-core contraction (stage ii,
 * Eq. 16 term (ii), on split-BF16 tables) of a plan built with
 * PAT_FLAG_BF16_SPLIT (default 2; 0 = always the CUDA-core path). PAT_ERR_ARG
 * for a negative min_batch; PAT_ERR_UNSUPPORTED for min_batch > 0 on a plan
 * without split-BF16 tables. */
int pat_plan_set_tensor_batch(pat_plan* plan, int min_batch);

/* Measurement operator (Sec. 2.3, Sec. 3.3): the object stays on the
 * reconstruction grid while the data are recorded only at the scan positions
 *   x = ox + sx i (0 <= i < mx),  y = oy + sy j (0 <= j < my),
 *   mx = ceil((nx - ox) / sx),    my = ceil((ny - oy) / sy),
 * of the nx x ny sensor grid (e.g. sx = sy = 2 for a reconstruction grid twice
 * as fine as the scan grid). Afterwards pat_forward applies S H (H of Eq. 7-8,
 * then keep the scan positions; data real_t[batch][nt][my][mx]), pat_adjoint
 * applies H* S^T (zero-fill the other sensor positions, then Eq. 11), and
 * pat_gradient, pat_power_norm, pat_fista_solve and the slots use that pair.
 * sx = sy = 1, ox = oy = 0 restores the plain operator. Needs sx, sy >= 1,
 * 0 <= ox < nx, 0 <= oy < ny. Synchronises the device; the plan's cached
 * graphs are rebuilt on next use and data loaded into slots must be reloaded.
 * The diagnostic stage entry points are not affected. */
int pat_plan_set_sampling(pat_plan* plan, int sx, int sy, int ox, int oy);

/* Folds the sensors' temporal impulse response into the resident library
 * (Sec. 2: identical, spatially invariant sensor responses incorporated into
 * the kernels by temporal convolution): every kernel becomes
 *   h'_z(., t) = sum_{tau = 0 .. min(nr - 1, t)} r[tau] h_z(., t - tau),
 * causal, r[0] at lag 0, over the recorded samples t < nt, so H' rho is H rho
 * convolved with r along time at every sensor position. r: host double[nr],
 * nr >= 1. Calls compose (two calls fold the convolution of both responses).
 * The split-BF16 tiles, if any, are rebuilt. pat_plan_info's table statistics
 * keep describing the library as built. Synchronises `stream`. */
int pat_plan_set_sensor_response(pat_plan* plan, const double* r, int nr, pat_stream stream);

/* Synchronises the device and reports whether any bounded device-side wait of
 * the plan's kernels gave up since the last check (PAT_ERR_TIMEOUT; the flag
 * is cleared), else PAT_OK. */
int pat_plan_check(pat_plan* plan);

/* Limit of the pipeline waits of the tensor-core contraction (the mbarrier
 * waits between its table stream, operand staging, MMAs and accumulator
 * drain): each tests its barrier at most `polls` times (< 2^32; each test may
 * suspend the thread for a short, hardware-defined time) before the kernel
 * gives up: it then records the timeout for pat_plan_check, lets every copy
 * and MMA it has issued finish (bounded by 2 s of device time), frees its
 * tensor memory and returns, leaving that call's output undefined. polls < 0
 * restores the default PAT_WAIT_LIMIT_DEFAULT (a few seconds per wait);
 * polls = 0 makes every pipeline wait give up at once, which exercises that
 * path without a device fault. Synchronises the device; cached graphs are
 * rebuilt on next use. Not described in the paper (a property of this
 * implementation's kernels). */
#define PAT_WAIT_LIMIT_DEFAULT 4194304
int pat_plan_set_wait_limit(pat_plan* plan, int64_t polls);

/* Device allocations the library currently holds over all plans (diagnostic:
 * a failed pat_plan_create* leaves this count unchanged). Setting the
 * environment variable PAT_DEBUG_FAIL_ALLOC = n (n >= 1) before a
 * pat_plan_create* call makes the n-th device allocation of that call fail as
 * if the device were out of memory (PAT_ERR_OOM), to test the clean-up path;
 * unset it for normal use. */
int64_t pat_debug_live_allocations(void);

/* --- operators ----------------------------------------------------------------- */

/* d = H rho (Eq. 7-8) for `batch` volumes. rho: real_t[batch][nz][ny][nx] in,
 * d: real_t[batch][nt][ny][nx] out. 1 <= batch <= max_batch. */
int pat_forward(pat_plan* plan, const void* rho, void* d, int batch, pat_stream stream);

/* rho = H* d (Eq. 11), the exact transpose of pat_forward under the Euclidean
 * inner products of Eq. 10. */
int pat_adjoint(pat_plan* plan, const void* d, void* rho, int batch, pat_stream stream);

/* Gradient of the data term, Eq. 15: grad = H*(H x - y). x, grad:
 * real_t[batch][nz][ny][nx]; y: real_t[batch][nt][ny][nx]. If resid2 is not
 * NULL, *resid2 (host) receives ||H x - y||^2 summed over the batch
 * (FP64 accumulation) and the call synchronises `stream`. */
int pat_gradient(pat_plan* plan, const void* x, const void* y, void* grad, int batch,
                 double* resid2, pat_stream stream);

/* L = ||H*H||_2 by power iteration (not printed in the paper; FISTA's step):
 * v <- H*H v / ||H*H v|| from the start vector v0 (real_t[nz][ny][nx], host or
 * device, need not be normalised), `iters` >= 1 steps; *L_out (host) =
 * ||H*H v|| of the last step. Norms accumulate in FP64. Synchronises `stream`. */
int pat_power_norm(pat_plan* plan, const void* v0, int iters, double* L_out,
                   pat_stream stream);

/* pat_power_norm (the step-size constant L of Eq. 12-14; not printed in the
 * paper) from a seeded start vector generated on the device:
 *   v0[i] = 2 u_i - 1,  u_i = (splitmix64(seed + (i + 1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53,
 * i = 0 .. nz*ny*nx - 1 in the object's memory order (x fastest), splitmix64
 * the finaliser of Steele, Lea & Flood (2014): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
 * z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31; then rounded to real_t.
 * The same generator is what pat_fista_solve uses (seed 0x5EED) when it
 * estimates L itself. Synchronises `stream`. */
int pat_power_norm_seed(pat_plan* plan, int iters, uint64_t seed, double* L_out,
                        pat_stream stream);

/* FISTA for Eq. 12 with f of Eq. 13 and g of Eq. 14, per volume:
 *   y_1 = x_0, t_1 = 1;  x_k = max(y_k - (H*(H y_k - d))/L - lambda/L, 0);
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;
 *   y_{k+1} = x_k + ((t_k - 1)/t_{k+1}) (x_k - x_{k-1}).
 * y: measured data real_t[batch][nt][ny][nx]; x: real_t[batch][nz][ny][nx],
 * read when warm_start = 1, overwritten with x_iters. Each iteration runs as
 * one replay of a CUDA graph captured on the first call for this batch size.
 * `report` may be NULL; if given, the call synchronises `stream` and fills it. */
int pat_fista_solve(pat_plan* plan, const void* y, void* x, int batch,
                    const pat_fista_params* params, pat_fista_report* report,
                    pat_stream stream);

/* <a, b> = sum_i a[i] b[i] with products and sums in FP64 (the adjoint test of
 * Eq. 9 and the norms). a, b: real_t[n] device arrays of the plan's precision.
 * *out (host) receives the result; synchronises `stream`. Deterministic: the
 * same inputs give the same bits. */
int pat_dot_f64(pat_plan* plan, const void* a, const void* b, int64_t n, double* out,
                pat_stream stream);

/* --- continuous batching: FISTA requests in slots --------------------------------- */

/* A plan's max_batch slots each hold one FISTA reconstruction in progress
 * (Eq. 12-14): its measured data, x_{k-1}, momentum point y_k and its own
 * t_k, beta_k, 1/L, lambda/L, iteration count and last residual norm. Requests
 * enter and leave between steps, so the slots sit at different iterations.
 * pat_slots_step(n) advances slots [0, n) by one FISTA iteration each: one
 * batched H (the table is read once per group of volumes instead of once per
 * request), one batched H*, and each slot's own prox/momentum update; every
 * step is one CUDA graph, captured the first time this n is used. The
 * iterates are those of pat_fista_solve run on the request alone.
 * All calls are stream-ordered on `stream`. */

/* Loads a request into `slot`: copies y (real_t[nt][ny][nx], host or device;
 * a host y has been copied when the call returns), sets x_0 = y_1 = 0,
 * t_1 = 1, and the step 1/L and weight lambda (L > 0, lambda >= 0). */
int pat_slot_load(pat_plan* plan, int slot, const void* y, double lambda, double L,
                  pat_stream stream);

/* Copies the whole state of slot `src` into slot `dst` (to keep the active
 * requests packed in [0, n) when one leaves). */
int pat_slot_move(pat_plan* plan, int dst, int src, pat_stream stream);

/* One FISTA iteration for slots [0, n), 0 <= n <= max_batch. If `kernels` is
 * not NULL it receives the kernel launches of the step. */
int pat_slots_step(pat_plan* plan, int n, int* kernels, pat_stream stream);

/* Copies the current iterate x_k of `slot` (real_t[nz][ny][nx]) to x (host or
 * device; may be NULL) and, if resid2 is not NULL, ||H y_k - d||^2 of its last
 * step to *resid2 (host; the call then synchronises `stream`). */
int pat_slot_read(pat_plan* plan, int slot, void* x, double* resid2, pat_stream stream);

/* --- diagnostics: the FFT stages on their own ----------------------------------- */

/* Zero-pads `slices` real [ny][nx] slices to py x px and applies the 2D real
 * DFT (stage i of Sec. 3.2; Eq. 16 term (i)). Output in the plan's spectral
 * layout: complex[slices][px/2 + 1][py] (kx-major, ky contiguous).
 * in: real_t[slices][ny][nx] device; out: device. slices <= max_batch * max(nz, nt). */
int pat_stage_spectrum(pat_plan* plan, const void* in, void* out, int slices,
                       pat_stream stream);

/* Inverse of the layout above for `slices` planes: unnormalised inverse 2D DFT
 * (sum over k of X(k) exp(+2 pi i k.n / P)), real part, cropped to [ny][nx]
 * (stage iii; Eq. 16 term (iii)). */
int pat_stage_image(pat_plan* plan, const void* in, void* out, int slices,
                    pat_stream stream);

/* Stage ii alone (Eq. 16 term (ii)): the per-frequency contraction with the
 * resident table, on device arrays of complex real_t with row stride
 * bins_padded and bin index k = kx * py + ky (kx in [0, px/2]):
 *   adjoint = 0:  out[b][t][k] = sum_z Hh[k][t][z] in[b][z][k]        (Eq. 7)
 *   adjoint = 1:  out[b][z][k] = sum_t conj(Hh[k][t][z]) in[b][t][k]  (Eq. 11)
 * Hh carries the 1/(px py) factor of the inverse transform. */
int pat_stage_contract(pat_plan* plan, const void* in, void* out, int batch, int adjoint,
                       pat_stream stream);

/* --- frequency shards: the operator split over ranks --------------------------------- */

/* Stage ii (Eq. 16 term (ii), the per-frequency contraction) is independent
 * per frequency bin, so `world` ranks (one per GPU) can each keep an equal
 * share of the table's rows (D4 representatives of a folded library, else
 * bins): the stored operator, whose size is the limitation discussed in
 * Sec. 4, then scales as 1 / world per GPU. Stages i and iii are split by
 * slices: rank r holds depth slices [r nz/world, (r+1) nz/world) of objects
 * and time samples [r nt/world, (r+1) nt/world) of data. One all-to-all of
 * slice spectra sits at each stage boundary (the caller runs it, e.g.
 * NCCL all_to_all_single on equal chunks):
 *   H:  pat_shard_spectrum(side 0, rho_r) -> send[world][nz/world][W]
 *       all-to-all                         -> X[nz][W]  (this rank's slots of every depth)
 *       pat_shard_contract(0, X)           -> Y[nt][W]  = [world][nt/world][W]
 *       all-to-all                         -> recv[world][nt/world][W]
 *       pat_shard_image(side 1, recv)      -> d_r [nt/world][ny][nx]
 *   H*: the same with sides and directions swapped.
 * Spectra are complex float; W = slot_width: the rank's rows times 4 slots
 * per representative (folded) or 1 per bin. Slots no bin uses are never read.
 * Requires world | nz and world | nt. */
typedef struct {
  int32_t world, rank;
  int32_t nz_local, nt_local; /* slices of this rank: nz / world, nt / world */
  int32_t folded;             /* 1: rows are D4 representatives */
  int32_t reserved;
  int64_t rows_total;         /* table rows of the whole operator */
  int64_t rows_per_rank;      /* equal range per rank, a multiple of 32 */
  int64_t row0, rows;         /* this rank's rows [row0, row0 + rows) */
  int64_t slot_width;         /* W: complex values per exchange row */
  int64_t bins;               /* frequency bins (px/2 + 1) py */
} pat_shard_info;

/* Host only (no device call): the block layout of the CUDA-core contraction
 * of a folded P x P plan (D4 representatives u as enumerated by the library:
 * a = 0..P/2, b = a..P/2, representative (kx, ky) = (a, b), up to 4 bins).
 * The table is stored as chunks of 32 rows; block j of the contraction reads
 * chunk rb_chunk[j], and its lane l handles representative rb_rep[32 j + l]
 * (-1 = none) with the spectra of stored row 32 rb_chunk[j] + l. With
 * `radial` = 0 block j reads chunk j and handles representatives 32 j ..
 * 32 j + 31. With `radial` = 1 representatives are grouped by a^2 + b^2: the
 * m representatives of a radius sit at the same lane of m consecutive blocks
 * that share one chunk, whose row holds the spectra of the radius's first
 * representative (the blocks' table reads coincide, so the stored table shrinks
 * by the shared rows); when that would not store fewer chunks than the
 * identity layout (small P: every group size pads its last chunk) the identity
 * layout is returned. Outputs: *nrb blocks, *nch chunks, and (optional, host
 * arrays) rb_rep[32 nrb], rb_chunk[nrb], row_rep[32 nch] (representative
 * whose spectra fill each stored row, -1 = unused) and rep_row[U] (stored row
 * of each representative, U = (P/2 + 1)(P/2 + 2) / 2). Call with NULL arrays
 * to get the sizes. PAT_ERR_ARG for P not a supported even length. */
int pat_fold_blocks(int P, int radial, int64_t* nrb, int64_t* nch, int32_t* rb_rep,
                    int32_t* rb_chunk, int32_t* row_rep, int32_t* rep_row);

/* Host only (no device call): the partition of rank `rank` of `world` for a
 * library stored folded (`fold` = 1) or per bin (stage ii is independent per
 * frequency bin, Eq. 16 term (ii); splitting its rows divides the stored
 * operator of Sec. 4 over the ranks). Optional outputs (host
 * arrays): zmap[bins] / tmap[bins], the position of every bin k of one slice
 * in the depth-side / time-side exchange buffer (owner q of k's row:
 * q * (slices per rank) * W + slot of k), and members_local[rows_per_rank * 4]
 * (folded: slot of member i of this rank's j-th representative, -1 = none). */
int pat_shard_layout(const pat_geometry* g, int fold, int rank, int world, pat_shard_info* info,
                     int32_t* zmap, int32_t* tmap, int32_t* members_local);

/* A plan holding only this rank's rows of the library generated from `m`
 * (as pat_plan_create_kspace; single precision, max_batch = 1). It runs only
 * the pat_shard_* stages (other operator entry points return PAT_ERR_ARG).
 * Its workspace holds no spectra, object or data buffers (the exchange
 * buffers are the caller's): twiddles, the FFT intermediate of
 * max(nz, nt) / world slices, reduction scratch and scalars. */
int pat_plan_create_kspace_shard(const pat_geometry* g, const pat_medium* m, int rank, int world,
                                 pat_stream stream, pat_plan** out);
/* The partition of a shard plan (as pat_shard_layout); PAT_ERR_ARG for a plan
 * that is not a shard. No device call. */
int pat_plan_shard_info(const pat_plan* plan, pat_shard_info* info);

/* Stage i of this rank's slices (side 0: depth slices of an object, side 1:
 * time samples of data; in float[n][ny][nx], n = nz_local or nt_local) into
 * the send buffer complex[world][n][W] (Eq. 16 term (i)). Device arrays. */
int pat_shard_spectrum(pat_plan* plan, int side, const float* in, void* send, pat_stream stream);

/* Stage ii on this rank's rows: adjoint = 0: in X[nz][W] -> out Y[nt][W]
 * (Eq. 7); adjoint = 1: in D[nt][W] -> out Z[nz][W] (Eq. 11). */
int pat_shard_contract(pat_plan* plan, int adjoint, const void* in, void* out, pat_stream stream);

/* Stage iii of this rank's slices from the received spectra
 * recv[world][n][W] into out float[n][ny][nx] (Eq. 16 term (iii)). With
 * `sub` (same shape as out): out = image - sub, and if r2 is not NULL *r2
 * (host) = sum of out^2 in FP64 over this rank's slices (the call then
 * synchronises `stream`). */
int pat_shard_image(pat_plan* plan, int side, const void* recv, float* out, const float* sub,
                    double* r2, pat_stream stream);

/* The FISTA update of Eq. 14-15 on n device floats (a distributed solve keeps
 * each rank's depth slices): x = max(y - grad invL - lamL, 0),
 * y <- x + beta (x - xprev), xprev <- x. */
int pat_fista_step(float* y, float* xprev, const float* grad, int64_t n, double invL, double lamL,
                   double beta, pat_stream stream);

/* y = a x + b y on n device floats (x may equal y): the scaling and
 * combination steps of a distributed power iteration (the L of Eq. 12-14) or
 * data synthesis. */
int pat_axpby(float* y, const float* x, int64_t n, double a, double b, pat_stream stream);

/* Stage ii of the folded split-BF16 path as the operator runs it, on spectra
 * already in its representative-slot layout (no conversion): rows of
 * 4 * ceil(U / 32) * 32 complex float, bin k at slot 4 u + i (member i of its
 * D4 representative u), in[b][nz or nt][row], out likewise. Only for plans
 * built with PAT_FLAG_BF16_SPLIT, folded, and batch >= the tensor batch
 * (PAT_ERR_ARG otherwise). Eq. 16 term (ii); a timing aid for the tensor-core
 * contraction alone. */
int pat_stage_contract_slots(pat_plan* plan, const void* in, void* out, int batch, int adjoint,
                             pat_stream stream);

/* --- for callers that cannot allocate device memory ----------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory at the point of the call (an application
 * whose device memory is owned by its own pool allocator, or a latency-critical
 * loop where cudaMalloc, which can synchronise the device, is not allowed).
 *
 * Same result as pat_stage_spectrum, without a plan and without allocating:
 * zero-pads `slices` real float [ny][nx] slices (in, device) to py x px and
 * writes their 2D real DFT to out (device), complex float [slices][px/2+1][py].
 * Both arrays must be on the calling thread's current device (PAT_ERR_ARG
 * otherwise); the work runs there, on `stream`, which must belong to it.
 * The row-pass intermediate lives in a static device array of 64 MiB that
 * every GPU loading the library holds until the process exits; requests with
 * slices * (px/2 + 1) * (ny rounded up to even) * 8 > 64 MiB return
 * PAT_ERR_ARG. No cudaMalloc, cudaFree or allocating library call is made.
 * The first call on a device sets that device up (symbol lookup and a
 * synchronous twiddle upload): make it before any stream capture. All calls
 * share the static array (it keeps the last call's contents; nothing in it has
 * to start at zero), so calls that overlap on the GPU race: serialise them on
 * one stream. px, py: powers of two in [16, 1024], px >= 2nx - 1, py >= 2ny - 1. */
int pat_spectrum_noalloc(const float* in, int nx, int ny, int px, int py, int slices,
                         void* out, pat_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* PAT_H */
