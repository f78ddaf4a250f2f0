// C ABI of libpat (declared in include/pat.h): plans, the operator H (Eq. 7-8),
// its adjoint H* (Eq. 11), the gradient of Eq. 15, the power iteration for
// ||H*H|| and FISTA (Eq. 12-14) composed from the stage kernels.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "pat_internal.h"

namespace pat {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PAT_ERR_OOM : PAT_ERR_CUDA;
}

static std::atomic<int64_t> g_live_allocs{0};
static thread_local long g_fail_countdown = 0;  // 0: no injected failure pending

cudaError_t dev_alloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  if (g_fail_countdown > 0 && --g_fail_countdown == 0) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}
void dev_free(void* p) {
  if (p && cudaFree(p) == cudaSuccess) g_live_allocs.fetch_sub(1);
}
void alloc_hook_arm() {
  const char* v = std::getenv("PAT_DEBUG_FAIL_ALLOC");
  const long n = v ? std::strtol(v, nullptr, 10) : 0;
  g_fail_countdown = n > 0 ? n : 0;
}
void alloc_hook_disarm() { g_fail_countdown = 0; }

}  // namespace pat

using namespace pat;

namespace {

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

int validate(const pat_geometry* g) {
  if (!g) return fail(PAT_ERR_ARG, "geometry is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nt < 1)
    return fail(PAT_ERR_ARG, "nx, ny, nz, nt must be >= 1");
  if (!fft_len_ok(g->px) || !fft_len_ok(g->py))
    return fail(PAT_ERR_UNSUPPORTED, "px and py must be 2^k or 3*2^k in [16, 1024]");
  if (g->px < 2 * g->nx - 1 || g->py < 2 * g->ny - 1)
    return fail(PAT_ERR_ARG, "padding too small for linear convolution: need px >= 2nx-1, py >= 2ny-1");
  if (g->max_batch < 1) return fail(PAT_ERR_ARG, "max_batch must be >= 1");
  if (g->flags & ~(PAT_FLAG_FP64 | PAT_FLAG_FORCE_COMPLEX | PAT_FLAG_BF16_SPLIT | PAT_FLAG_NO_FOLD |
                   PAT_FLAG_NO_RADIAL))
    return fail(PAT_ERR_ARG, "unknown flags");
  const int64_t smax = (int64_t)g->max_batch * std::max(g->nz, g->nt);
  if (smax > 65535) return fail(PAT_ERR_UNSUPPORTED, "max_batch * max(nz, nt) must be <= 65535");
  return PAT_OK;
}

Layout make_layout(const pat_geometry* g) {
  Layout L{};
  L.nx = g->nx;
  L.ny = g->ny;
  L.nz = g->nz;
  L.nt = g->nt;
  L.px = g->px;
  L.py = g->py;
  L.max_batch = g->max_batch;
  L.fp64 = (g->flags & PAT_FLAG_FP64) != 0;
  L.rsize = L.fp64 ? 8 : 4;
  L.K = (int64_t)(g->px / 2 + 1) * g->py;
  L.Kpad = (L.K + 31) / 32 * 32;
  L.nkb = L.Kpad / 32;
  L.tstride = g->ny + (g->ny & 1);
  L.tslice = (int64_t)(g->px / 2 + 1) * L.tstride;
  L.mx = g->nx;
  L.my = g->ny;
  set_representation(L, false);
  return L;
}

void free_plan(pat_plan* pp) {
  if (!pp) return;
  Plan& p = pp->p;
  PlanExt& x = pp->x;
  for (Graph* g = p.graphs; g;) {
    Graph* n = g->next;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    g = n;
  }
  // the plan's own memory: the table side, buffers allocated on first use,
  // and the workspace arena unless the caller owns it
  void* owned[] = {p.table,      p.tc_fwd,     p.tc_adj,     p.fold_members, p.fold_rep,
                   p.fold_slot,  p.rb_members, p.rb_chunk,   p.rep_row,      p.shard_zmap,
                   p.shard_tmap, p.shard_members};
  for (void* b : owned) dev_free(b);
  if (x.io_heap) {
    dev_free(x.io_obj[0]);
    dev_free(x.io_obj[1]);
    dev_free(x.io_dat);
  }
  if (p.hist_heap) {
    dev_free(p.betas);
    dev_free(p.r2_dev);
  }
  if (!p.ws_external) dev_free(p.ws_base);
  if (x.cap) cudaStreamDestroy(x.cap);
  delete pp;
}

// Fills the twiddle tables exp(-2 pi i k / n) (already carved from the workspace).
int upload_twiddles(Plan& p) {
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < 2; ++a) {
    const int n = a == 0 ? p.L.px : p.L.py;
    std::vector<double> w(2 * (size_t)n);
    for (int k = 0; k < n; ++k) {
      w[2 * k] = std::cos(-2.0 * pi * k / n);
      w[2 * k + 1] = std::sin(-2.0 * pi * k / n);
    }
    void* dst = a == 0 ? p.twx : p.twy;
    if (p.L.fp64) {
      PAT_CUDA(cudaMemcpy(dst, w.data(), w.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> f(w.begin(), w.end());
      PAT_CUDA(cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
  }
  return PAT_OK;
}

// Upper bound of the blocks of the stage-iii row kernel (its residual partials).
int c2r_partials_bound(const Layout& L) {
  const int64_t smax = (int64_t)L.max_batch * std::max(L.nz, L.nt);
  return (int)(smax * ((L.ny + 1) / 2 + 1));
}

// Complex elements per row of the X / Y spectra buffers: the bins (Kpad), or
// the representative slots 4 * Upad of a folded single-precision plan's
// batched tensor-core path, whichever is longer.
int64_t spectrum_row_cap(const Layout& L) {
  if (L.fp64 || L.px != L.py) return L.Kpad;
  const int64_t h = L.px / 2, U = (h + 1) * (h + 2) / 2;
  return std::max<int64_t>(L.Kpad, 4 * ((U + 31) / 32 * 32));
}

// FISTA momentum / residual history kept in the workspace: 4096 iterations
// per solve (a plan that allocates its own memory grows it on demand).
constexpr int kHistCap = 4097;
constexpr size_t kWsAlign = 256;

// Walks the workspace regions of a plan in their fixed order, each aligned to
// 256 bytes; with `base` the plan's pointers are set to their regions.
// `with_io` adds the host-pointer staging buffers. `lean_slices` > 0 gives
// the arena of a frequency shard, whose spectra are the caller's exchange
// buffers: only the twiddles, an FFT intermediate of that many slices, the
// reduction scratch and the scalars (every other pointer stays NULL).
// Returns the bytes spanned.
size_t ws_walk(pat_plan* pp, unsigned char* base, bool with_io, int64_t lean_slices = 0) {
  Plan& p = pp->p;
  PlanExt& x = pp->x;
  const Layout& L = p.L;
  const bool lean = lean_slices > 0;
  const size_t cs = 2 * L.rsize;
  const int64_t smax = lean ? lean_slices : (int64_t)L.max_batch * std::max(L.nz, L.nt);
  const size_t xy = lean ? 0 : (size_t)smax * spectrum_row_cap(L) * cs;
  const size_t tb = (size_t)smax * L.tslice * cs;
  const size_t vol = lean ? 0 : (size_t)L.max_batch * L.nz * L.ny * L.nx * L.rsize;
  const size_t dat = lean ? 0 : (size_t)L.max_batch * L.nt * L.ny * L.nx * L.rsize;
  const int partials = std::max(kReduceBlocks, c2r_partials_bound(L));
  const size_t sb = lean ? 0 : sizeof(double) * L.max_batch;
  const int hist = lean ? 0 : kHistCap;
  size_t off = 0;
  auto take = [&](auto** dst, size_t bytes) {
    if (base) {
      *dst = bytes ? reinterpret_cast<std::remove_pointer_t<decltype(dst)>>(base + off) : nullptr;
    }
    off += (bytes + kWsAlign - 1) / kWsAlign * kWsAlign;
  };
  take(&p.twx, (size_t)L.px * cs);
  take(&p.twy, (size_t)L.py * cs);
  take(&p.X, xy);
  take(&p.Y, xy);
  take(&p.T, tb);
  take(&p.vol_a, vol);
  take(&p.vol_b, vol);
  take(&p.vol_c, vol);
  take(&p.dat_a, dat);
  take(&p.dat_b, dat);
  take(&p.red, sizeof(double) * partials);
  take(&x.res, sizeof(double) * 8);
  take(&x.scal, sizeof(double) * 2);
  take(&p.iter_dev, 3 * sizeof(int));
  take(&x.slots.t, sb);
  take(&x.slots.beta, sb);
  take(&x.slots.invL, sb);
  take(&x.slots.lamL, sb);
  take(&x.slots.r2, sb);
  take(&x.slots.k, lean ? 0 : sizeof(int) * L.max_batch);
  take(&p.betas, sizeof(double) * hist);
  take(&p.r2_dev, sizeof(double) * hist);
  take(&p.tc_err, sizeof(int));
  if (with_io && !lean) {
    take(&x.io_obj[0], vol);
    take(&x.io_obj[1], vol);
    take(&x.io_dat, dat);
  }
  if (base) {
    x.c2r_partials = partials;
    p.betas_cap = p.r2_cap = hist;
  }
  return off;
}

// Device bytes of a plan's workspace for layout L (with_io: including the
// host-pointer staging buffers).
int64_t workspace_bytes(const Layout& L, bool with_io) {
  pat_plan tmp;
  tmp.p.L = L;
  return (int64_t)ws_walk(&tmp, nullptr, with_io);
}

// Carves the workspace from `user` (caller-owned device memory of ws_bytes)
// or from one block the plan allocates, and initialises what must start at
// zero or at fixed values.
int setup_workspace(pat_plan* pp, void* user, size_t ws_bytes, int64_t lean_slices = 0) {
  Plan& p = pp->p;
  const bool ext = user != nullptr;
  const size_t need = ws_walk(pp, nullptr, ext, lean_slices);
  if (ext) {
    if (!is_device_ptr(user)) return fail(PAT_ERR_ARG, "workspace is not device memory");
    if (reinterpret_cast<uintptr_t>(user) % kWsAlign)
      return fail(PAT_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < need)
      return fail(PAT_ERR_ARG, "workspace smaller than pat_workspace_size: need " +
                                   std::to_string(need) + " bytes");
    p.ws_base = static_cast<unsigned char*>(user);
    p.ws_external = true;
  } else {
    PAT_CUDA(dev_alloc(&p.ws_base, need));
  }
  p.ws_cap = ext ? ws_bytes : need;
  p.ws_used = ws_walk(pp, p.ws_base, ext, lean_slices);
  p.ws_bytes = p.ws_used;
  PAT_CUDA(cudaMemset(p.iter_dev, 0, 3 * sizeof(int)));
  PAT_CUDA(cudaMemset(p.tc_err, 0, sizeof(int)));
  PAT_CUDA(cudaStreamCreateWithFlags(&pp->x.cap, cudaStreamNonBlocking));
  return upload_twiddles(p);
}

int ensure_io(pat_plan* pp) {
  PlanExt& x = pp->x;
  if (x.io_dat) return PAT_OK;
  const Layout& L = pp->p.L;
  const size_t vol = (size_t)L.max_batch * L.nz * L.ny * L.nx * L.rsize;
  const size_t dat = (size_t)L.max_batch * L.nt * L.ny * L.nx * L.rsize;
  x.io_heap = true;
  PAT_CUDA(dev_alloc(&x.io_obj[0], vol));
  PAT_CUDA(dev_alloc(&x.io_obj[1], vol));
  PAT_CUDA(dev_alloc(&x.io_dat, dat));
  pp->p.ws_bytes += 2 * vol + dat;
  return PAT_OK;
}

// Arms the allocation fault injector for the duration of a plan creation.
struct AllocHook {
  AllocHook() { alloc_hook_arm(); }
  ~AllocHook() { alloc_hook_disarm(); }
};

int create_common(const pat_geometry* g, void* ws, size_t ws_bytes, pat_plan** out,
                  pat_plan** pp_out, int64_t lean_slices = 0) {
  if (!out) return fail(PAT_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(g);
  if (rc != PAT_OK) return rc;
  pat_plan* pp = new (std::nothrow) pat_plan();
  if (!pp) return fail(PAT_ERR_OOM, "host allocation of the plan failed");
  pp->p.L = make_layout(g);
  pp->p.tc_spin = kTcSpinDefault;
  if ((rc = setup_workspace(pp, ws, ws_bytes, lean_slices)) != PAT_OK) {
    free_plan(pp);
    return rc;
  }
  *pp_out = pp;
  return PAT_OK;
}

// Split-BF16 tensor-core tables (PAT_FLAG_BF16_SPLIT), from the real table.
int build_tensor_tables(pat_plan* pp, int flags, cudaStream_t s) {
  if (!(flags & PAT_FLAG_BF16_SPLIT)) return PAT_OK;
  Plan& p = pp->p;
  if (!tc_supported(p.L))
    return fail(PAT_ERR_UNSUPPORTED,
                "PAT_FLAG_BF16_SPLIT needs a real single-precision table, nz = 128 and nt a "
                "multiple of 128 up to 512");
  const size_t one = tc_table_bytes(p.L);
  PAT_CUDA(dev_alloc(&p.tc_fwd, one));
  PAT_CUDA(dev_alloc(&p.tc_adj, one));
  PAT_CUDA(tc_build_tables(p, p.tc_fwd, p.tc_adj, s));
  PAT_CUDA(cudaStreamSynchronize(s));
  p.tc_bytes = 2 * one;
  p.tc_min_batch = 2;
  return PAT_OK;
}

// Destroys the cached CUDA graphs (they captured pointers and launch
// parameters that are about to change).
void drop_graphs(Plan& p) {
  for (Graph* g = p.graphs; g;) {
    Graph* n = g->next;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    g = n;
  }
  p.graphs = nullptr;
}

size_t obj_elems(const Layout& L, int batch) { return (size_t)batch * L.nz * L.ny * L.nx; }
// data live on the scan grid (the whole sensor grid unless sampling is set)
size_t dat_elems(const Layout& L, int batch) { return (size_t)batch * L.nt * L.my * L.mx; }

}  // namespace

namespace pat {

cudaError_t forward_dev(const Plan& p, const void* rho, void* d, int batch, cudaStream_t s,
                        const void* sub, double* sumsq, int groups, double* group_sums) {
  const Layout& L = p.L;
  const int64_t plane = (int64_t)L.ny * L.nx, scan = (int64_t)L.my * L.mx;
  const bool sl = tc_slots(p, batch);
  const int64_t row = sl ? slot_row(L) : L.Kpad;
  const int* slot = sl ? p.fold_slot : nullptr;
  cudaError_t e = launch_spectrum(p, rho, plane, L.nx, L.ny, p.X, row, batch * L.nz, s,
                                  no_sampling(), slot);
  if (e != cudaSuccess) return e;
  if ((e = launch_contract_fwd(p, p.X, p.Y, batch, s)) != cudaSuccess) return e;
  return launch_image(p, p.Y, row, d, scan, batch * L.nt, sub, sumsq, s, groups, group_sums,
                      sampling_of(L), slot);
}

cudaError_t gradient_dev(const Plan& p, const void* x, const void* y, void* grad, int batch,
                         cudaStream_t s, double* sumsq, int groups, double* group_sums,
                         const FistaStep* step) {
  const Layout& L = p.L;
  const int64_t plane = (int64_t)L.ny * L.nx, scan = (int64_t)L.my * L.mx;
  const bool sl = tc_slots(p, batch);
  const int64_t row = sl ? slot_row(L) : L.Kpad;
  const int* slot = sl ? p.fold_slot : nullptr;
  // with a step that leaves the row transform of the next x in T, stage i
  // here is its column pass alone
  cudaError_t e = (step && step->next_T)
                      ? launch_spectrum_cols(p, L.ny, p.X, row, batch * L.nz, s, slot)
                      : launch_spectrum(p, x, plane, L.nx, L.ny, p.X, row, batch * L.nz, s,
                                        no_sampling(), slot);
  if (e != cudaSuccess) return e;
  if ((e = launch_contract_fwd(p, p.X, p.Y, batch, s)) != cudaSuccess) return e;
  if ((e = launch_residual(p, p.Y, row, y, scan, batch * L.nt, sumsq, s, groups, group_sums,
                           sampling_of(L), slot, p.Y, row)) != cudaSuccess)
    return e;
  if ((e = launch_contract_adj(p, p.Y, p.X, batch, s)) != cudaSuccess) return e;
  if (step) return launch_image_step(p, p.X, row, batch * L.nz, *step, s, slot);
  return launch_image(p, p.X, row, grad, plane, batch * L.nz, nullptr, nullptr, s, 0, nullptr,
                      no_sampling(), slot);
}

cudaError_t adjoint_dev(const Plan& p, const void* d, void* rho, int batch, cudaStream_t s) {
  const Layout& L = p.L;
  const int64_t plane = (int64_t)L.ny * L.nx, scan = (int64_t)L.my * L.mx;
  const bool sl = tc_slots(p, batch);
  const int64_t row = sl ? slot_row(L) : L.Kpad;
  const int* slot = sl ? p.fold_slot : nullptr;
  cudaError_t e = launch_spectrum(p, d, scan, L.nx, L.ny, p.Y, row, batch * L.nt, s,
                                  sampling_of(L), slot);
  if (e != cudaSuccess) return e;
  if ((e = launch_contract_adj(p, p.Y, p.X, batch, s)) != cudaSuccess) return e;
  return launch_image(p, p.X, row, rho, plane, batch * L.nz, nullptr, nullptr, s, 0, nullptr,
                      no_sampling(), slot);
}

cudaError_t instantiate_counted(cudaGraph_t graph, cudaGraphExec_t* exec, int* kernels) {
  size_t n = 0;
  *kernels = 0;
  cudaError_t e = cudaGraphGetNodes(graph, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e == cudaSuccess && n) e = cudaGraphGetNodes(graph, nodes.data(), &n);
  for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
      ++*kernels;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
  return e;
}

}  // namespace pat

namespace {

int check_call(pat_plan* plan, int batch) {
  if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
  if (plan->p.shard_world)
    return fail(PAT_ERR_ARG, "a frequency-shard plan runs only the pat_shard_* stages");
  if (batch < 0 || batch > plan->p.L.max_batch)
    return fail(PAT_ERR_ARG, "batch must be in [0, max_batch]");
  return PAT_OK;
}

// Host-or-device argument: a device pointer is used as is; a host pointer is
// staged (copied in for inputs) through `stage`.
struct Arg {
  const void* user;
  void* dev;
  bool host;
};

int stage_in(Arg& a, void* stage, size_t bytes, cudaStream_t s) {
  a.host = !is_device_ptr(a.user);
  a.dev = a.host ? stage : const_cast<void*>(a.user);
  if (a.host && bytes) PAT_CUDA(cudaMemcpyAsync(stage, a.user, bytes, cudaMemcpyHostToDevice, s));
  return PAT_OK;
}

int any_host(std::initializer_list<const void*> ptrs) {
  for (const void* q : ptrs)
    if (q && !is_device_ptr(q)) return 1;
  return 0;
}

// Seeded start vector of the power iteration (splitmix64 of Steele, Lea &
// Flood 2014 on the counter seed + (i + 1) * golden gamma -> uniform [-1, 1));
// any start with a component along the top singular vector works.
template <typename R>
__global__ void k_fill_hash(R* v, int64_t n, unsigned long long seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (R)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

int fill_seeded(pat_plan* pp, uint64_t seed, cudaStream_t s) {
  Plan& p = pp->p;
  const int64_t n = (int64_t)obj_elems(p.L, 1);
  if (p.L.fp64)
    k_fill_hash<double><<<64, 256, 0, s>>>(static_cast<double*>(p.vol_a), n, seed);
  else
    k_fill_hash<float><<<64, 256, 0, s>>>(static_cast<float*>(p.vol_a), n, seed);
  PAT_CUDA(cudaGetLastError());
  return PAT_OK;
}

// Power iteration on the plan's buffers: v in vol_a (normalised here first).
int power_dev(pat_plan* pp, int iters, double* L_out, cudaStream_t s) {
  Plan& p = pp->p;
  PlanExt& x = pp->x;
  const Layout& L = p.L;
  const int64_t n = (int64_t)obj_elems(L, 1);
  PAT_CUDA(launch_dot(p, p.vol_a, p.vol_a, n, x.res + 2, s));
  PAT_CUDA(launch_scale_by_inv_norm(p, p.vol_a, p.vol_a, n, x.res + 2, s));
  for (int i = 0; i < iters; ++i) {
    PAT_CUDA(forward_dev(p, p.vol_a, p.dat_a, 1, s));
    PAT_CUDA(adjoint_dev(p, p.dat_a, p.vol_c, 1, s));
    PAT_CUDA(launch_dot(p, p.vol_c, p.vol_c, n, x.res + 2, s));
    PAT_CUDA(launch_scale_by_inv_norm(p, p.vol_c, p.vol_a, n, x.res + 2, s));
  }
  double h = 0;
  PAT_CUDA(cudaMemcpyAsync(&h, x.res + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  PAT_CUDA(cudaStreamSynchronize(s));
  *L_out = std::sqrt(h);
  return PAT_OK;
}

// One FISTA iteration on the plan's buffers (what the graph holds):
// vol_a = y_k, vol_b = x_{k-1}, dat_b = measured data.
cudaError_t fista_iter(pat_plan* pp, int batch, cudaStream_t s) {
  Plan& p = pp->p;
  PlanExt& x = pp->x;
  // the gradient's last stage applies the step in place (no gradient array)
  const FistaStep step{p.vol_a, p.vol_b, x.scal, p.betas, p.iter_dev, x.res + 1, p.r2_dev,
                       p.r2_cap, reinterpret_cast<unsigned*>(p.iter_dev + 1), true};
  return gradient_dev(p, p.vol_a, p.dat_b, nullptr, batch, s, x.res + 1, 0, nullptr, &step);
}

Graph* graph_for(pat_plan* pp, int batch, int* rc) {
  Plan& p = pp->p;
  for (Graph* g = p.graphs; g; g = g->next)
    if (g->kind == 0 && g->batch == batch) return g;
  cudaStream_t cs = pp->x.cap;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t e2 = fista_iter(pp, batch, cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (e2 != cudaSuccess) e = e2;
  }
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  if (e == cudaSuccess) e = instantiate_counted(graph, &exec, &kernels);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "capturing the FISTA iteration graph");
    return nullptr;
  }
  Graph* g = new (std::nothrow) Graph();
  if (!g) {
    cudaGraphExecDestroy(exec);
    *rc = fail(PAT_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  g->batch = batch;
  g->kernels = kernels;
  g->exec = exec;
  g->next = p.graphs;
  p.graphs = g;
  return g;
}

}  // namespace

namespace pat {
int plan_create_common(const pat_geometry* g, pat_plan** out, pat_plan** pp,
                       int64_t lean_slices) {
  return create_common(g, nullptr, 0, out, pp, lean_slices);
}
void plan_free(pat_plan* pp) { free_plan(pp); }
}  // namespace pat


#define PAT_GUARD_BEGIN try {
#define PAT_GUARD_END                                                  \
  }                                                                    \
  catch (const std::bad_alloc&) {                                      \
    return fail(PAT_ERR_OOM, "host allocation failed");                \
  }                                                                    \
  catch (...) {                                                        \
    return fail(PAT_ERR_CUDA, "unexpected internal error");            \
  }

extern "C" {

const char* pat_last_error(void) { return pat::g_err.c_str(); }

int pat_plan_create_with_workspace(const pat_geometry* g, const void* table, pat_table_format fmt,
                                   void* workspace, size_t ws_bytes, pat_stream stream,
                                   pat_plan** out) {
  PAT_GUARD_BEGIN
  AllocHook hook;
  if (!table) return fail(PAT_ERR_ARG, "table is NULL");
  if (fmt < PAT_TABLE_SPATIAL_F64 || fmt > PAT_TABLE_SPECTRAL_C64)
    return fail(PAT_ERR_ARG, "unknown table format");
  pat_plan* pp = nullptr;
  int rc = create_common(g, workspace, ws_bytes, out, &pp);
  if (rc != PAT_OK) return rc;
  rc = build_table_from_source(pp->p, table, fmt, (g->flags & PAT_FLAG_FORCE_COMPLEX) != 0,
                               (g->flags & PAT_FLAG_NO_FOLD) == 0,
                               (g->flags & PAT_FLAG_NO_RADIAL) == 0, (cudaStream_t)stream);
  if (rc == PAT_OK) rc = build_tensor_tables(pp, g->flags, (cudaStream_t)stream);
  if (rc != PAT_OK) {
    free_plan(pp);
    return rc;
  }
  *out = pp;
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_create(const pat_geometry* g, const void* table, pat_table_format fmt,
                    pat_stream stream, pat_plan** out) {
  return pat_plan_create_with_workspace(g, table, fmt, nullptr, 0, stream, out);
}

int pat_plan_create_kspace_with_workspace(const pat_geometry* g, const pat_medium* m,
                                          void* workspace, size_t ws_bytes, pat_stream stream,
                                          pat_plan** out) {
  PAT_GUARD_BEGIN
  AllocHook hook;
  if (!m) return fail(PAT_ERR_ARG, "medium is NULL");
  if (!(m->c > 0 && m->dx > 0 && m->dy > 0 && m->dz > 0 && m->dt > 0))
    return fail(PAT_ERR_ARG, "medium: c, dx, dy, dz, dt must be > 0");
  if (m->z0 < 0 || !pow2_in(m->mz, 2, 1 << 16) || m->mz <= m->z0 + (g ? g->nz : 0))
    return fail(PAT_ERR_ARG, "medium: mz must be a power of two > z0 + nz, z0 >= 0");
  pat_plan* pp = nullptr;
  int rc = create_common(g, workspace, ws_bytes, out, &pp);
  if (rc != PAT_OK) return rc;
  rc = build_table_kspace(pp->p, *m, (g->flags & PAT_FLAG_FORCE_COMPLEX) != 0,
                          (g->flags & PAT_FLAG_NO_FOLD) == 0,
                          (g->flags & PAT_FLAG_NO_RADIAL) == 0, (cudaStream_t)stream);
  if (rc == PAT_OK) rc = build_tensor_tables(pp, g->flags, (cudaStream_t)stream);
  if (rc != PAT_OK) {
    free_plan(pp);
    return rc;
  }
  *out = pp;
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_create_kspace(const pat_geometry* g, const pat_medium* m, pat_stream stream,
                           pat_plan** out) {
  return pat_plan_create_kspace_with_workspace(g, m, nullptr, 0, stream, out);
}

int64_t pat_workspace_size(const pat_geometry* g) {
  PAT_GUARD_BEGIN
  const int rc = validate(g);
  if (rc != PAT_OK) return rc;
  return workspace_bytes(make_layout(g), true);
  PAT_GUARD_END
}

int64_t pat_debug_live_allocations(void) { return g_live_allocs.load(); }

int pat_plan_set_wait_limit(pat_plan* plan, int64_t polls) {
  PAT_GUARD_BEGIN
  if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
  if (polls > 0xFFFFFFFFll) return fail(PAT_ERR_ARG, "polls must be < 2^32");
  const int64_t v = polls < 0 ? kTcSpinDefault : polls;
  if (v != plan->p.tc_spin) {
    // the cached graphs hold the old limit in their kernel parameters
    PAT_CUDA(cudaDeviceSynchronize());
    drop_graphs(plan->p);
    plan->p.tc_spin = v;
  }
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_destroy(pat_plan* plan) {
  PAT_GUARD_BEGIN
  if (!plan) return PAT_OK;
  cudaDeviceSynchronize();
  free_plan(plan);
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_estimate(const pat_geometry* g, int real_table, int64_t* table_bytes,
                      int64_t* workspace) {
  PAT_GUARD_BEGIN
  int rc = validate(g);
  if (rc != PAT_OK) return rc;
  if (!table_bytes || !workspace) return fail(PAT_ERR_ARG, "output pointer is NULL");
  if (real_table < 0 || real_table > 3) return fail(PAT_ERR_ARG, "real_table must be 0..3");
  Layout L = make_layout(g);
  set_representation(L, real_table != 0);
  if (real_table >= 2 && fold_possible(L)) {  // D4-folded, radially shared with 3
    std::vector<int> members, rep, slot;
    fold_enumerate(L.px, members, rep, slot);
    L.U = (int64_t)members.size() / 4;
    L.Upad = (L.U + 31) / 32 * 32;
    L.nub = L.Upad / 32;
    FoldBlocks fb;
    fold_blocks(L.px, members, L.U, real_table == 3, fb);
    L.nrb = fb.nrb;
    L.nch = fb.nch;
    L.radial = fb.nch != fb.nrb;
    set_representation(L, true, true);
  }
  *table_bytes = (int64_t)L.table_bytes;
  if ((g->flags & PAT_FLAG_BF16_SPLIT) && tc_supported(L))
    *table_bytes += 2 * (int64_t)tc_table_bytes(L);
  *workspace = workspace_bytes(L, true);
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_info(const pat_plan* plan, pat_plan_info_t* info) {
  if (!plan || !info) return fail(PAT_ERR_ARG, "plan or info is NULL");
  const Plan& p = plan->p;
  info->real_table = p.L.real ? 1 : 0;
  info->fp64 = p.L.fp64 ? 1 : 0;
  info->bins = p.L.K;
  info->bins_padded = p.L.Kpad;
  info->table_bytes = (int64_t)p.L.table_bytes;
  info->workspace_bytes = (int64_t)p.ws_bytes;
  info->workspace_external = p.ws_external ? 1 : 0;
  info->table_max_abs = p.table_max_abs;
  info->table_max_imag = p.table_max_imag;
  info->tensor_table_bytes = (int64_t)p.tc_bytes;
  info->tensor_min_batch = p.tc_fwd ? p.tc_min_batch : 0;
  info->folded = p.L.fold ? 1 : 0;
  info->table_rows = p.L.fold ? p.L.U : p.L.K;
  info->radial = p.L.fold && p.L.radial ? 1 : 0;
  // every stored row takes nt z-groups of 16 bytes, whatever the representation
  info->stored_rows = (int64_t)(p.L.table_bytes / ((size_t)p.L.nt * p.L.nzg * 16));
  return PAT_OK;
}

int pat_plan_set_tensor_batch(pat_plan* plan, int min_batch) {
  if (!plan || min_batch < 0) return fail(PAT_ERR_ARG, "plan is NULL or min_batch < 0");
  if (!plan->p.tc_fwd && min_batch > 0)
    return fail(PAT_ERR_UNSUPPORTED, "plan has no split-BF16 tables (PAT_FLAG_BF16_SPLIT)");
  plan->p.tc_min_batch = min_batch;
  return PAT_OK;
}

int pat_plan_set_sampling(pat_plan* plan, int sx, int sy, int ox, int oy) {
  PAT_GUARD_BEGIN
  if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
  Layout& L = plan->p.L;
  if (sx < 1 || sy < 1 || ox < 0 || oy < 0 || ox >= L.nx || oy >= L.ny)
    return fail(PAT_ERR_ARG, "need sx, sy >= 1 and 0 <= ox < nx, 0 <= oy < ny");
  // work queued on the plan's buffers must not see the layout change
  PAT_CUDA(cudaDeviceSynchronize());
  drop_graphs(plan->p);
  L.sx = sx;
  L.sy = sy;
  L.ox = ox;
  L.oy = oy;
  L.mx = (L.nx - ox + sx - 1) / sx;
  L.my = (L.ny - oy + sy - 1) / sy;
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_set_sensor_response(pat_plan* plan, const double* r, int nr, pat_stream stream) {
  PAT_GUARD_BEGIN
  if (!plan || !r || nr < 1) return fail(PAT_ERR_ARG, "need a plan, r != NULL and nr >= 1");
  if (is_device_ptr(r)) return fail(PAT_ERR_ARG, "r must be host memory");
  Plan& p = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = apply_sensor_response(p, r, nr, s);
  if (rc != PAT_OK) return rc;
  if (p.tc_fwd) {  // the split-BF16 tiles follow the table
    PAT_CUDA(tc_build_tables(p, p.tc_fwd, p.tc_adj, s));
    PAT_CUDA(cudaStreamSynchronize(s));
  }
  return PAT_OK;
  PAT_GUARD_END
}

int pat_plan_check(pat_plan* plan) {
  PAT_GUARD_BEGIN
  if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
  PAT_CUDA(cudaDeviceSynchronize());
  int h = 0;
  PAT_CUDA(cudaMemcpy(&h, plan->p.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    PAT_CUDA(cudaMemset(plan->p.tc_err, 0, sizeof(int)));
    return fail(PAT_ERR_TIMEOUT, "a bounded wait of the tensor-core contraction gave up");
  }
  return PAT_OK;
  PAT_GUARD_END
}

int pat_forward(pat_plan* plan, const void* rho, void* d, int batch, pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, batch);
  if (rc != PAT_OK) return rc;
  if (batch == 0) return PAT_OK;
  if (!rho || !d) return fail(PAT_ERR_ARG, "rho or d is NULL");
  Plan& p = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = obj_elems(p.L, batch) * p.L.rsize, db = dat_elems(p.L, batch) * p.L.rsize;
  if (any_host({rho, d}) && (rc = ensure_io(plan)) != PAT_OK) return rc;
  Arg a{rho, nullptr, false};
  if ((rc = stage_in(a, plan->x.io_obj[0], ob, s)) != PAT_OK) return rc;
  const bool hout = !is_device_ptr(d);
  void* dst = hout ? plan->x.io_dat : d;
  PAT_CUDA(forward_dev(p, a.dev, dst, batch, s));
  if (hout) {
    PAT_CUDA(cudaMemcpyAsync(d, dst, db, cudaMemcpyDeviceToHost, s));
    PAT_CUDA(cudaStreamSynchronize(s));
  } else if (a.host) {
    PAT_CUDA(cudaStreamSynchronize(s));
  }
  return PAT_OK;
  PAT_GUARD_END
}

int pat_adjoint(pat_plan* plan, const void* d, void* rho, int batch, pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, batch);
  if (rc != PAT_OK) return rc;
  if (batch == 0) return PAT_OK;
  if (!rho || !d) return fail(PAT_ERR_ARG, "rho or d is NULL");
  Plan& p = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = obj_elems(p.L, batch) * p.L.rsize, db = dat_elems(p.L, batch) * p.L.rsize;
  if (any_host({rho, d}) && (rc = ensure_io(plan)) != PAT_OK) return rc;
  Arg a{d, nullptr, false};
  if ((rc = stage_in(a, plan->x.io_dat, db, s)) != PAT_OK) return rc;
  const bool hout = !is_device_ptr(rho);
  void* dst = hout ? plan->x.io_obj[0] : rho;
  PAT_CUDA(adjoint_dev(p, a.dev, dst, batch, s));
  if (hout) {
    PAT_CUDA(cudaMemcpyAsync(rho, dst, ob, cudaMemcpyDeviceToHost, s));
    PAT_CUDA(cudaStreamSynchronize(s));
  } else if (a.host) {
    PAT_CUDA(cudaStreamSynchronize(s));
  }
  return PAT_OK;
  PAT_GUARD_END
}

int pat_gradient(pat_plan* plan, const void* xin, const void* y, void* grad, int batch,
                 double* resid2, pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, batch);
  if (rc != PAT_OK) return rc;
  if (batch == 0) {
    if (resid2) *resid2 = 0.0;
    return PAT_OK;
  }
  if (!xin || !y || !grad) return fail(PAT_ERR_ARG, "x, y or grad is NULL");
  Plan& p = plan->p;
  PlanExt& px = plan->x;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = obj_elems(p.L, batch) * p.L.rsize, db = dat_elems(p.L, batch) * p.L.rsize;
  if (any_host({xin, y, grad}) && (rc = ensure_io(plan)) != PAT_OK) return rc;
  Arg ax{xin, nullptr, false}, ay{y, nullptr, false};
  if ((rc = stage_in(ax, px.io_obj[0], ob, s)) != PAT_OK) return rc;
  if ((rc = stage_in(ay, px.io_dat, db, s)) != PAT_OK) return rc;
  const bool hout = !is_device_ptr(grad);
  void* dst = hout ? px.io_obj[1] : grad;
  PAT_CUDA(gradient_dev(p, ax.dev, ay.dev, dst, batch, s, px.res + 1));
  if (hout) PAT_CUDA(cudaMemcpyAsync(grad, dst, ob, cudaMemcpyDeviceToHost, s));
  if (resid2) PAT_CUDA(cudaMemcpyAsync(resid2, px.res + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (hout || resid2 || ax.host || ay.host) PAT_CUDA(cudaStreamSynchronize(s));
  return PAT_OK;
  PAT_GUARD_END
}

int pat_power_norm(pat_plan* plan, const void* v0, int iters, double* L_out, pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, 1);
  if (rc != PAT_OK) return rc;
  if (!v0 || !L_out || iters < 1) return fail(PAT_ERR_ARG, "v0 / L_out NULL or iters < 1");
  Plan& p = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = obj_elems(p.L, 1) * p.L.rsize;
  PAT_CUDA(cudaMemcpyAsync(p.vol_a, v0, ob, cudaMemcpyDefault, s));
  return power_dev(plan, iters, L_out, s);
  PAT_GUARD_END
}

int pat_power_norm_seed(pat_plan* plan, int iters, uint64_t seed, double* L_out,
                        pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, 1);
  if (rc != PAT_OK) return rc;
  if (!L_out || iters < 1) return fail(PAT_ERR_ARG, "L_out NULL or iters < 1");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = fill_seeded(plan, seed, s)) != PAT_OK) return rc;
  return power_dev(plan, iters, L_out, s);
  PAT_GUARD_END
}

int pat_fista_solve(pat_plan* plan, const void* y, void* x, int batch,
                    const pat_fista_params* prm, pat_fista_report* report, pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, batch);
  if (rc != PAT_OK) return rc;
  if (!y || !x || !prm) return fail(PAT_ERR_ARG, "y, x or params is NULL");
  if (prm->iters < 0 || !(prm->lambda >= 0) || (prm->L <= 0 && prm->power_iters < 1))
    return fail(PAT_ERR_ARG, "need iters >= 0, lambda >= 0, and L > 0 or power_iters >= 1");
  Plan& p = plan->p;
  PlanExt& px = plan->x;
  const Layout& L = p.L;
  cudaStream_t s = (cudaStream_t)stream;
  double Lc = prm->L;
  if (Lc <= 0) {
    if ((rc = fill_seeded(plan, 0x5EEDull, s)) != PAT_OK) return rc;
    if ((rc = power_dev(plan, prm->power_iters, &Lc, s)) != PAT_OK) return rc;
    Lc *= 1.01;
  }
  if (batch == 0) {
    if (report) *report = pat_fista_report{Lc, 0, 0, 0, 0};
    return PAT_OK;
  }
  const size_t ob = obj_elems(L, batch) * L.rsize, db = dat_elems(L, batch) * L.rsize;
  // momentum coefficients beta_k = (t_k - 1) / t_{k+1} (FP64 on the host)
  const int iters = prm->iters;
  if (p.betas_cap < iters + 1) {
    if (p.ws_external)
      return fail(PAT_ERR_ARG, "a plan on caller-owned workspace runs at most " +
                                   std::to_string(p.betas_cap - 1) + " FISTA iterations per call");
    // grow the history outside the workspace (graphs captured the old pointers)
    PAT_CUDA(cudaStreamSynchronize(s));
    drop_graphs(p);
    if (p.hist_heap) {
      dev_free(p.betas);
      dev_free(p.r2_dev);
    }
    p.betas = nullptr;
    p.r2_dev = nullptr;
    p.betas_cap = p.r2_cap = 0;
    p.hist_heap = true;
    const int cap = iters + 1;
    PAT_CUDA(dev_alloc(&p.betas, sizeof(double) * cap));
    PAT_CUDA(dev_alloc(&p.r2_dev, sizeof(double) * cap));
    p.betas_cap = p.r2_cap = cap;
  }
  std::vector<double> betas(iters + 1, 0.0);
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    betas[k] = (t - 1.0) / tn;
    t = tn;
  }
  const double scal[2] = {1.0 / Lc, prm->lambda / Lc};
  PAT_CUDA(cudaMemcpyAsync(p.betas, betas.data(), sizeof(double) * (iters + 1),
                           cudaMemcpyHostToDevice, s));
  PAT_CUDA(cudaMemcpyAsync(px.scal, scal, sizeof(scal), cudaMemcpyHostToDevice, s));
  PAT_CUDA(cudaMemsetAsync(p.iter_dev, 0, sizeof(int), s));
  PAT_CUDA(cudaMemsetAsync(p.r2_dev, 0, sizeof(double) * p.r2_cap, s));
  PAT_CUDA(cudaMemcpyAsync(p.dat_b, y, db, cudaMemcpyDefault, s));
  if (prm->warm_start) {
    PAT_CUDA(cudaMemcpyAsync(p.vol_b, x, ob, cudaMemcpyDefault, s));
    PAT_CUDA(cudaMemcpyAsync(p.vol_a, p.vol_b, ob, cudaMemcpyDeviceToDevice, s));
  } else {
    PAT_CUDA(cudaMemsetAsync(p.vol_b, 0, ob, s));
    PAT_CUDA(cudaMemsetAsync(p.vol_a, 0, ob, s));
  }
  int kernels_per_iter = 0;
  if (iters > 0) {
    Graph* g = graph_for(plan, batch, &rc);
    if (!g) return rc;
    // stage i's row transform of y_1 into T; each iteration's step kernel
    // leaves the next one there
    PAT_CUDA(launch_spectrum_rows(p, p.vol_a, (int64_t)L.ny * L.nx, L.nx, L.ny, batch * L.nz, s));
    kernels_per_iter = g->kernels;
    for (int k = 0; k < iters; ++k) PAT_CUDA(cudaGraphLaunch(g->exec, s));
  }
  PAT_CUDA(cudaMemcpyAsync(x, p.vol_b, ob, cudaMemcpyDefault, s));
  if (report) {
    double r2[2] = {0, 0};
    if (iters > 0) {
      PAT_CUDA(cudaMemcpyAsync(&r2[0], p.r2_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      PAT_CUDA(cudaMemcpyAsync(&r2[1], p.r2_dev + (iters - 1), sizeof(double),
                               cudaMemcpyDeviceToHost, s));
    }
    PAT_CUDA(cudaStreamSynchronize(s));
    *report = pat_fista_report{Lc, r2[0], r2[1], iters, kernels_per_iter};
  } else if (!is_device_ptr(x)) {
    PAT_CUDA(cudaStreamSynchronize(s));
  }
  return PAT_OK;
  PAT_GUARD_END
}

int pat_dot_f64(pat_plan* plan, const void* a, const void* b, int64_t n, double* out,
                pat_stream stream) {
  PAT_GUARD_BEGIN
  if (!plan || !a || !b || !out || n < 0) return fail(PAT_ERR_ARG, "bad dot arguments");
  if (n > 0 && (!is_device_ptr(a) || !is_device_ptr(b)))
    return fail(PAT_ERR_ARG, "pat_dot_f64 takes device arrays");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    *out = 0.0;
    return PAT_OK;
  }
  PAT_CUDA(launch_dot(plan->p, a, b, n, plan->x.res, s));
  PAT_CUDA(cudaMemcpyAsync(out, plan->x.res, sizeof(double), cudaMemcpyDeviceToHost, s));
  PAT_CUDA(cudaStreamSynchronize(s));
  return PAT_OK;
  PAT_GUARD_END
}

int pat_stage_spectrum(pat_plan* plan, const void* in, void* out, int slices, pat_stream stream) {
  PAT_GUARD_BEGIN
  if (!plan || !in || !out) return fail(PAT_ERR_ARG, "bad arguments");
  if (plan->p.shard_world) return fail(PAT_ERR_ARG, "a frequency-shard plan runs only the pat_shard_* stages");
  const Layout& L = plan->p.L;
  if (slices < 0 || slices > L.max_batch * std::max(L.nz, L.nt))
    return fail(PAT_ERR_ARG, "slices must be in [0, max_batch * max(nz, nt)]");
  PAT_CUDA(launch_spectrum(plan->p, in, (int64_t)L.ny * L.nx, L.nx, L.ny, out, L.K, slices,
                           (cudaStream_t)stream));
  return PAT_OK;
  PAT_GUARD_END
}

int pat_stage_image(pat_plan* plan, const void* in, void* out, int slices, pat_stream stream) {
  PAT_GUARD_BEGIN
  if (!plan || !in || !out) return fail(PAT_ERR_ARG, "bad arguments");
  if (plan->p.shard_world) return fail(PAT_ERR_ARG, "a frequency-shard plan runs only the pat_shard_* stages");
  const Layout& L = plan->p.L;
  if (slices < 0 || slices > L.max_batch * std::max(L.nz, L.nt))
    return fail(PAT_ERR_ARG, "slices must be in [0, max_batch * max(nz, nt)]");
  PAT_CUDA(launch_image(plan->p, in, L.K, out, (int64_t)L.ny * L.nx, slices, nullptr, nullptr,
                        (cudaStream_t)stream));
  return PAT_OK;
  PAT_GUARD_END
}

int pat_stage_contract(pat_plan* plan, const void* in, void* out, int batch, int adjoint,
                       pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, batch);
  if (rc != PAT_OK) return rc;
  if (batch == 0) return PAT_OK;
  if (!in || !out) return fail(PAT_ERR_ARG, "in or out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const Plan& p = plan->p;
  const int64_t rin = (int64_t)batch * (adjoint ? p.L.nt : p.L.nz);
  const int64_t rout = (int64_t)batch * (adjoint ? p.L.nz : p.L.nt);
  if (tc_slots(p, batch)) {  // the tensor path's slot layout, converted in and out
    PAT_CUDA(launch_to_slots(p, in, p.X, rin, s));
    if (adjoint)
      PAT_CUDA(launch_contract_adj(p, p.X, p.Y, batch, s));
    else
      PAT_CUDA(launch_contract_fwd(p, p.X, p.Y, batch, s));
    PAT_CUDA(launch_from_slots(p, p.Y, out, rout, s));
    return PAT_OK;
  }
  if (adjoint)
    PAT_CUDA(launch_contract_adj(p, in, out, batch, s));
  else
    PAT_CUDA(launch_contract_fwd(p, in, out, batch, s));
  return PAT_OK;
  PAT_GUARD_END
}

int pat_stage_contract_slots(pat_plan* plan, const void* in, void* out, int batch, int adjoint,
                             pat_stream stream) {
  PAT_GUARD_BEGIN
  int rc = check_call(plan, batch);
  if (rc != PAT_OK) return rc;
  if (batch == 0) return PAT_OK;
  if (!in || !out) return fail(PAT_ERR_ARG, "in or out is NULL");
  const Plan& p = plan->p;
  if (!tc_slots(p, batch))
    return fail(PAT_ERR_ARG, "the representative-slot layout belongs to the folded split-BF16 "
                             "path at batch >= its tensor batch");
  cudaStream_t s = (cudaStream_t)stream;
  if (adjoint)
    PAT_CUDA(launch_contract_adj(p, in, out, batch, s));
  else
    PAT_CUDA(launch_contract_fwd(p, in, out, batch, s));
  return PAT_OK;
  PAT_GUARD_END
}

}  // extern "C"
