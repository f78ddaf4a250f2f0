// Internal declarations shared by the CUDA translation units of libpat.
// Not part of the public ABI (that is include/pat.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pat.h"

namespace pat {

// Transverse transform lengths the FFT stages support: 2^k or 3 * 2^k in
// [16, 1024].
inline bool fft_len_ok(int v) {
  if (v < 16 || v > 1024) return false;
  if (v % 3 == 0) v /= 3;
  return (v & (v - 1)) == 0;
}

// ----------------------------------------------------------------------------
// Complex numbers in registers / memory: (x = re, y = im), 8 or 16 bytes.
// ----------------------------------------------------------------------------
template <typename R>
struct cx;
template <>
struct __align__(8) cx<float> {
  float x, y;
};
template <>
struct __align__(16) cx<double> {
  double x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return mk<R>(a.x + b.x, a.y + b.y);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
  return mk<R>(a.x - b.x, a.y - b.y);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> conjg(cx<R> a) {
  return mk<R>(a.x, -a.y);
}

// 16-byte vector of the table stream.
template <typename R>
struct vec16;
template <>
struct vec16<float> {
  typedef float4 type;
};
template <>
struct vec16<double> {
  typedef double2 type;
};

// ----------------------------------------------------------------------------
// Plan: geometry, resident table, workspace.
// ----------------------------------------------------------------------------
// Frequency bins: k = kx * py + ky with kx in [0, px/2], ky in [0, py)
// ("kx-major half spectrum"); K = (px/2 + 1) py, padded to Kpad (multiple of 32).
// Table: [kb = k / 32][t][zg][lane = k % 32][ZG] elements, 16 bytes per
// (kb, t, zg, lane) group; ZG = z-planes per group (4 real f32, 2 complex f32
// or real f64, 1 complex f64).
struct Layout {
  int nx, ny, nz, nt, px, py, max_batch;
  bool fp64, real;
  int64_t K, Kpad, nkb;
  int zg, nzg;         // z per 16-byte group, number of groups
  int tstride;         // ny rounded up to even (row stride of the FFT intermediate)
  int64_t tslice;      // (px/2 + 1) * tstride
  size_t rsize;        // sizeof(real_t)
  size_t table_bytes;  // (fold ? nch : nkb) * nt * nzg * 32 * 16
  // D4 folding: the spectra depend only on {|kx|, |ky|}; one table row per
  // representative (a, b), 0 <= a <= b <= P/2, shared by up to 4 bins.
  bool fold = false;
  int64_t U = 0, Upad = 0, nub = 0;  // representatives, padded to 32, blocks of 32
  // Blocks of the CUDA-core contraction and stored chunks of 32 rows (equal
  // to nub without radial sharing; with it, the blocks of one radius group
  // share a chunk: representatives of equal a^2 + b^2 have one stored row).
  int64_t nrb = 0, nch = 0;
  bool radial = false;
  // Measurement operator: data live on the scan grid x = ox + sx i, y = oy + sy j
  // (i < mx, j < my) of the sensor grid; sx = sy = 1 is the plain operator.
  int sx = 1, sy = 1, ox = 0, oy = 0, mx = 0, my = 0;
};

// Sampling pattern handed to the row kernels (identity when s.on == false).
struct Samp {
  bool on;
  int sx, sy, ox, oy, mx, my;
};
inline Samp sampling_of(const Layout& L) {
  Samp s;
  s.on = L.sx != 1 || L.sy != 1 || L.ox != 0 || L.oy != 0;
  s.sx = L.sx;
  s.sy = L.sy;
  s.ox = L.ox;
  s.oy = L.oy;
  s.mx = L.mx;
  s.my = L.my;
  return s;
}
inline Samp no_sampling() { return Samp{false, 1, 1, 0, 0, 0, 0}; }

// ---- programmatic dependent launch ------------------------------------------
// The kernels of the operator and FISTA path are launched with launch_pdl: a
// kernel's blocks may be scheduled as the blocks of the previous kernel in its
// stream exit, do their prologue (index arithmetic, reads of plan constants
// such as twiddles and fold maps), then wait in pdl_wait() until the previous
// grid has completed and its writes are visible. Every kernel launched this
// way calls pdl_wait() before it touches any buffer that another kernel reads
// or writes. (Blocks do not signal their dependents early: measured on the
// bench geometry, an early signal let waiting blocks crowd the running
// contraction and cost more than the launch latency it hid.)
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- device allocations --------------------------------------------------------
// Every device allocation of a plan (its table, maps, workspace and the
// temporaries of table preparation) goes through dev_alloc / dev_free, which
// keep a count of live allocations (pat_debug_live_allocations). At the start
// of plan creation the environment variable PAT_DEBUG_FAIL_ALLOC = n (n >= 1)
// arms a host-side fault injector on the calling thread: the n-th allocation
// after that returns cudaErrorMemoryAllocation without allocating (testing the
// PAT_ERR_OOM and clean-up paths; no device fault involved).
cudaError_t dev_alloc_raw(void** p, size_t bytes);
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_raw(reinterpret_cast<void**>(p), bytes);
}
void dev_free(void* p);  // NULL is a no-op
void alloc_hook_arm();   // reads PAT_DEBUG_FAIL_ALLOC
void alloc_hook_disarm();

struct Graph;  // CUDA-graph cache (api.cu)

struct Plan {
  Layout L;
  double table_max_abs = 0, table_max_imag = 0;
  void* table = nullptr;  // device, blocked layout
  void* twx = nullptr;    // device cx<real_t>[px]: exp(-2 pi i k / px)
  void* twy = nullptr;    // device cx<real_t>[py]
  // workspace (device)
  void* X = nullptr;      // [max_batch][max(nz, nt)][Kpad] complex  (X or Z or D)
  void* Y = nullptr;      // [max_batch][max(nz, nt)][Kpad] complex  (Y or D or Z)
  void* T = nullptr;      // [max_batch * max(nz, nt)][tslice] complex
  void* vol_a = nullptr;  // [max_batch][nz][ny][nx] real: FISTA momentum point y_k
  void* vol_b = nullptr;  // [max_batch][nz][ny][nx] real: FISTA x_{k-1} / gradient
  void* vol_c = nullptr;  // [max_batch][nz][ny][nx] real: gradient
  void* dat_a = nullptr;  // [max_batch][nt][ny][nx] real: residual
  void* dat_b = nullptr;  // [max_batch][nt][ny][nx] real: measured data copy
  double* red = nullptr;  // reduction scratch: partials + results (see kReduce*)
  double* betas = nullptr;  // FISTA momentum coefficients per iteration
  int betas_cap = 0;
  bool hist_heap = false;   // betas / r2_dev were allocated outside the workspace
  int* iter_dev = nullptr;  // [0] FISTA iteration counter (graph replay), [1] block counter
                            // of the FISTA step pass, [2] block counter of the residual pass
  double* r2_dev = nullptr; // FISTA residual norms per iteration
  int r2_cap = 0;
  Graph* graphs = nullptr;
  size_t ws_bytes = 0;
  // Workspace arena: every per-call buffer above (twiddles, X, Y, T, the
  // object / data buffers, reductions, scalars, slot state, FISTA history, the
  // error flag of the tensor kernels, and the host-pointer staging when the
  // caller supplied the workspace) is carved from one block, either allocated
  // by the plan or owned by the caller (never freed by the plan).
  unsigned char* ws_base = nullptr;
  size_t ws_cap = 0, ws_used = 0;
  bool ws_external = false;
  // Pipeline wait limit of the tensor-core kernels (polls per wait).
  int64_t tc_spin = 0;
  // D4 folding maps (device): bins of each representative (-1 = none), and
  // the representative of each bin
  int* fold_members = nullptr;  // [Upad][4]
  int* fold_rep = nullptr;      // [K]
  // Slot layout of the spectra on the batched tensor-core path: row [Upad][4]
  // complex, bin k at fold_slot[k] = 4 u + i (the i-th member of its
  // representative u), so a representative's bins share one 32-byte sector.
  int* fold_slot = nullptr;     // [K]
  double fold_deviation = 0;    // max |Hh(bin) - Hh(representative)| seen (stored scale)
  double radial_deviation = 0;  // max |Hh(representative) - Hh(its stored row)| (user tables)
  // Block maps of the CUDA-core contraction (device): the bins of the
  // representative of each block slot (-1 = none), the stored chunk of each
  // block, and (radial plans) the stored row of each representative.
  int* rb_members = nullptr;    // [nrb * 32][4]
  int* rb_chunk = nullptr;      // [nrb]; NULL = block j reads chunk j
  int* rep_row = nullptr;       // [U]; NULL = representative u is row u
  // split-BF16 tensor-core tables (tc_contract.cu)
  void* tc_fwd = nullptr;
  void* tc_adj = nullptr;
  size_t tc_bytes = 0;   // both directions
  int* tc_err = nullptr; // device flag of timed-out waits
  int tc_min_batch = 0;
  // Frequency shard (pat_plan_create_kspace_shard): this plan holds table rows
  // [shard_row0, shard_row0 + shard_rows) of shard_world equal ranges of
  // shard_Wr rows; its spectra live in exchange buffers of rows of shard_W
  // complex values (4 slots per representative when folded, 1 per bin else).
  int shard_world = 0, shard_rank = 0;
  int64_t shard_row0 = 0, shard_rows = 0, shard_Wr = 0, shard_W = 0;
  int* shard_zmap = nullptr;     // [K] bin -> position in the depth-side exchange buffer
  int* shard_tmap = nullptr;     // [K] bin -> position in the time-side exchange buffer
  int* shard_members = nullptr;  // [Wr][4] local slots of this shard's representatives
};

constexpr int kReduceBlocks = 1024;  // max blocks of the FP64 reductions

// A captured iteration: FISTA (kind 0) or a slot step (kind 1) for `batch` volumes.
struct Graph {
  int kind = 0;
  int batch = 0;
  int kernels = 0;  // kernel nodes of the captured iteration
  cudaGraphExec_t exec = nullptr;
  Graph* next = nullptr;
};

// Per-slot FISTA state for continuous batching (device arrays of max_batch).
struct Slots {
  double* t = nullptr;     // t_k of the next iteration
  double* beta = nullptr;  // (t_k - 1) / t_{k+1}
  double* invL = nullptr;  // 1 / L
  double* lamL = nullptr;  // lambda / L
  double* r2 = nullptr;    // ||H y_k - d||^2 of the last step
  int* k = nullptr;        // iterations done
};

// Plan state beyond the operator: host-pointer staging, scalars, capture stream.
struct PlanExt {
  void* io_obj[2] = {nullptr, nullptr};  // host-pointer staging (objects)
  void* io_dat = nullptr;                // host-pointer staging (data)
  bool io_heap = false;                  // staging allocated on first use (not in the arena)
  double* res = nullptr;                 // device scalars: [0] dot, [1] r2 current, [2] norm
  double* scal = nullptr;                // device scalars: [0] 1/L, [1] lambda/L
  cudaStream_t cap = nullptr;            // private stream for graph capture
  int c2r_partials = 0;
  Slots slots;
};

struct FistaStep;  // below

// d = H rho / rho = H* d on device buffers of the plan's precision; with `sub`,
// the forward writes H rho - sub and sums its squares (FP64) into *sumsq, or,
// with groups > 0, per group of nt slices into group_sums[groups].
cudaError_t forward_dev(const Plan& p, const void* rho, void* d, int batch, cudaStream_t s,
                        const void* sub = nullptr, double* sumsq = nullptr, int groups = 0,
                        double* group_sums = nullptr);
cudaError_t adjoint_dev(const Plan& p, const void* d, void* rho, int batch, cudaStream_t s);
// grad = H*(S H x - y) (Eq. 15) with ||S H x - y||^2 summed into *sumsq, or per
// group of nt slices into group_sums[groups]; the residual stays on the chip.
cudaError_t gradient_dev(const Plan& p, const void* x, const void* y, void* grad, int batch,
                         cudaStream_t s, double* sumsq, int groups = 0,
                         double* group_sums = nullptr, const FistaStep* step = nullptr);
// Plan shell with its workspace (api.cu) and its release; lean_slices > 0
// gives a frequency shard's arena (no spectra, object or data buffers; an FFT
// intermediate of lean_slices slices).
int plan_create_common(const pat_geometry* g, pat_plan** out, pat_plan** pp,
                       int64_t lean_slices = 0);
void plan_free(pat_plan* pp);
// Records the kernel nodes of `graph`; instantiates it.
cudaError_t instantiate_counted(cudaGraph_t graph, cudaGraphExec_t* exec, int* kernels);

}  // namespace pat

struct pat_plan {
  pat::Plan p;
  pat::PlanExt x;
};

namespace pat {

// ----------------------------------------------------------------------------
// Error plumbing (thread-local message, status codes).
// ----------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PAT_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return pat::cuda_fail(e_, #call); \
  } while (0)

// ----------------------------------------------------------------------------
// Launchers (each returns cudaError_t of the launch).
// ----------------------------------------------------------------------------
// FFT stages. `in`/`out` element type follows L.fp64.
// Stage i: real slices [S][ny][nx] (slice stride in_stride elements, row
// length nx_in valid of px, ny_in valid rows of py) -> spectra [S][px/2+1][py]
// with slice stride out_stride complex elements.
cudaError_t launch_spectrum(const Plan& p, const void* in, int64_t in_stride, int nx_in, int ny_in,
                            void* out, int64_t out_stride, int S, cudaStream_t s,
                            Samp samp = no_sampling(), const int* slot = nullptr);
// Stage iii: spectra [S][px/2+1][py] -> real [S][ny][nx] (crop), optionally
// out = image - sub (sub has out's layout) with sum of squares added to
// *sumsq (FP64, via the plan's reduction scratch when sumsq != nullptr).
cudaError_t launch_image(const Plan& p, const void* in, int64_t in_stride, void* out,
                         int64_t out_stride, int S, const void* sub, double* sumsq,
                         cudaStream_t s, int groups = 0, double* group_sums = nullptr,
                         Samp samp = no_sampling(), const int* slot = nullptr);
// Stage iii then stage i on the data side of the gradient (Eq. 15): spectra
// of H x (rows of in_stride) -> spectra of r = S H x - y (rows of out_stride;
// out may be in), y [S][my][mx] with slice stride y_stride; ||r||^2 as in
// launch_image. The residual image is never stored.
cudaError_t launch_residual(const Plan& p, const void* in, int64_t in_stride, const void* y,
                            int64_t y_stride, int S, double* sumsq, cudaStream_t s, int groups,
                            double* group_sums, Samp samp, const int* slot, void* out,
                            int64_t out_stride);
// FISTA step (Eq. 14-15) fused into the last stage of the gradient: with g =
// H*(S H y_k - d) at a voxel, x_k = max(y_k - g/L - lambda/L, 0) and
// y_{k+1} = x_k + beta_k (x_k - x_{k-1}), scal = {1/L, lambda/L}, beta_k =
// betas[*iter] (device); y and xprev are updated in place. The last block to
// finish records r2_hist[*iter] = *r2_cur (if *iter < cap) and advances *iter
// (`done`: a zero-initialised block counter the kernel resets).
struct FistaStep {
  void* y;
  void* xprev;
  const double* scal;
  const double* betas;
  int* iter;
  const double* r2_cur;
  double* r2_hist;
  int cap;
  unsigned* done;
  bool next_T;  // also write the row transform of y_{k+1} over the rows of T
                // (the next iteration's stage i then runs its column pass only)
};
// Stage iii over the depth slices of `S` = batch * nz spectra with the FISTA
// step in place of the gradient store.
cudaError_t launch_image_step(const Plan& p, const void* in, int64_t in_stride, int S,
                              const FistaStep& f, cudaStream_t s, const int* slot);
// Stage i split in its two passes: rows of the real slices into the plan's T,
// and the column pass from T (launch_spectrum runs both).
cudaError_t launch_spectrum_rows(const Plan& p, const void* in, int64_t in_stride, int nx_in,
                                 int ny_in, int S, cudaStream_t s);
cudaError_t launch_spectrum_cols(const Plan& p, int ny_in, void* out, int64_t out_stride, int S,
                                 cudaStream_t s, const int* slot);
// Contractions over the resident table (tensor cores when the plan has the
// split tables and batch >= tc_min_batch).
cudaError_t launch_contract_fwd(const Plan& p, const void* X, void* Y, int batch, cudaStream_t s);
cudaError_t launch_contract_adj(const Plan& p, const void* D, void* Z, int batch, cudaStream_t s);

// The batched tensor-core contraction of a folded plan reads and writes
// spectra in the representative-slot layout (rows of 4 * Upad complex
// values, bin k at fold_slot[k]); every other path uses rows of Kpad bins.
inline bool tc_slots(const Plan& p, int batch) {
  return p.tc_fwd && p.L.fold && p.tc_min_batch > 0 && batch >= p.tc_min_batch;
}
inline int64_t slot_row(const Layout& L) { return 4 * L.Upad; }
// [S][Kpad] bins -> [S][4 Upad] slots and back (single precision).
cudaError_t launch_to_slots(const Plan& p, const void* in, void* out, int64_t S, cudaStream_t s);
cudaError_t launch_from_slots(const Plan& p, const void* in, void* out, int64_t S,
                              cudaStream_t s);
// Split-BF16 tensor-core contraction (tc_contract.cu).
bool tc_supported(const Layout& L);
size_t tc_table_bytes(const Layout& L);  // one direction
cudaError_t tc_build_tables(const Plan& p, void* fwd, void* adj, cudaStream_t s);
cudaError_t tc_contract(const Plan& p, const void* tables_fwd, const void* tables_adj,
                        const void* in, void* out, int batch, bool adjoint, int* err,
                        cudaStream_t s);
// Default pipeline wait limit of the tensor-core kernels (polls of
// mbarrier.try_wait per wait; a few seconds).
constexpr int64_t kTcSpinDefault = int64_t(1) << 22;

// Table construction (table.cu). Both allocate p.table and set the
// representation (real or complex) of p.L.
int build_table_from_source(Plan& p, const void* table, pat_table_format fmt, bool force_complex,
                            bool allow_fold, bool allow_radial, cudaStream_t s);
int build_table_kspace(Plan& p, const pat_medium& m, bool force_complex, bool allow_fold,
                       bool allow_radial, cudaStream_t s);
// Whether a k-space library of this layout is stored folded (real table on a
// square grid, dx = dy, single precision, folding allowed).
bool kspace_folds(const Layout& L, const pat_medium& m, bool allow_fold);
// Generates the k-space library rows at the given bins (one bin per table row,
// the row's representative when folded) into a newly allocated p.table of
// p.L.table_bytes in p.L's representation.
int kspace_generate(Plan& p, const pat_medium& m, const std::vector<int>& bins, cudaStream_t s);
// Host enumeration of the D4 representatives of a P x P half spectrum:
// members[4 u + i] (the up to 4 bins of representative u, -1 = none),
// rep[k] and slot[k] = 4 u + i for every bin k.
void fold_enumerate(int P, std::vector<int>& members, std::vector<int>& rep,
                    std::vector<int>& slot);
bool is_device_ptr(const void* p);
// Ordinal of the device holding `p`, or -1 if it is not device memory.
int device_of(const void* p);

// Representation-dependent parts of the layout.
inline void set_representation(Layout& L, bool real, bool fold = false) {
  L.real = real;
  L.fold = fold;
  const size_t esz = (L.fp64 ? 8 : 4) * (real ? 1 : 2);
  L.zg = (int)(16 / esz);
  L.nzg = (L.nz + L.zg - 1) / L.zg;
  L.table_bytes = (size_t)(fold ? L.nch : L.nkb) * L.nt * L.nzg * 32 * 16;
}

// D4 folding is possible for real single-precision tables on square padded
// grids (the symmetry itself is checked or guaranteed by the table builder).
inline bool fold_possible(const Layout& L) { return L.real && !L.fp64 && L.px == L.py; }
// Builds the folding maps of p (host enumeration, device copies) and sets
// L.U / Upad / nub; members (optional) receives the host copy of the
// representatives' bins [Upad][4].
int build_fold_maps(Plan& p, std::vector<int>* members);
// Block layout of the CUDA-core contraction of a folded table (see
// pat_fold_blocks): identity (one chunk per block) or radial sharing.
struct FoldBlocks {
  int64_t nrb = 0, nch = 0;
  std::vector<int> rb_rep;    // [nrb * 32] representative of each block slot, -1 = none
  std::vector<int> rb_chunk;  // [nrb] stored chunk of each block
  std::vector<int> row_rep;   // [nch * 32] representative filling each stored row, -1 = none
  std::vector<int> rep_row;   // [U] stored row of each representative
};
void fold_blocks(int P, const std::vector<int>& members, int64_t U, bool radial, FoldBlocks& fb);
// Sets L.nrb / nch / radial and uploads the block maps of `fb` to p.
int install_fold_blocks(Plan& p, const std::vector<int>& members, const FoldBlocks& fb);
// Folds the sensors' temporal response r[0..nr) into the resident table
// (causal convolution along time); synchronises `s`.
int apply_sensor_response(Plan& p, const double* r, int nr, cudaStream_t s);

// Vector kernels (vec.cu).
cudaError_t launch_dot(const Plan& p, const void* a, const void* b, int64_t n, double* out_dev,
                       cudaStream_t s);
// Sums n per-block partials (in order, FP64) into *out (device).
cudaError_t launch_partials_sum(const double* partials, int n, double* out, cudaStream_t s);
// out[g] = sum of partials[g * per, (g + 1) * per) for g < groups (in order, FP64).
cudaError_t launch_group_sums(const double* partials, int per, int groups, double* out,
                              cudaStream_t s);
cudaError_t launch_scale_by_inv_norm(const Plan& p, const void* in, void* out, int64_t n,
                                     const double* sumsq_dev, cudaStream_t s);

}  // namespace pat
