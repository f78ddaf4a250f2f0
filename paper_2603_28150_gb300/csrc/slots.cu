// Continuous batching of FISTA reconstructions (Eq. 12-15) on one plan.
//
// Each of a plan's max_batch slots holds one request in progress: its measured
// data (dat_b), x_{k-1} (vol_b), the momentum point y_k (vol_a), and its own
// scalars t_k, beta_k = (t_k - 1)/t_{k+1}, 1/L, lambda/L, iteration count and
// last residual norm. Requests join and leave between steps, so slots sit at
// different iterations; one step advances slots [0, n) together:
//   r = H y - d for all n volumes in one batched forward (the table is read
//       once per group of volumes, not once per request), per-slot ||r||^2;
//   g = H* r, batched;
//   per-slot prox + momentum update with that slot's own coefficients;
//   per-slot t_{k+1}, beta_{k+1} (FP64).
// The host keeps the active requests packed in [0, n) (pat_slot_move), and
// each step runs as a CUDA graph captured once per n.
#include <cmath>
#include <new>

#include "pat_internal.h"

namespace pat {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_slot_update(R* __restrict__ y, R* __restrict__ xprev,
                                                     const R* __restrict__ grad, int64_t vol,
                                                     int64_t n, const double* __restrict__ invL,
                                                     const double* __restrict__ lamL,
                                                     const double* __restrict__ beta) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / vol;
    const R yv = y[i], g = grad[i], xp = xprev[i];
    R x = yv - g * (R)invL[s] - (R)lamL[s];  // prox of Eq. 14 after the step of Eq. 15
    x = x > (R)0 ? x : (R)0;
    y[i] = x + (R)beta[s] * (x - xp);
    xprev[i] = x;
  }
}

// t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 and the next beta, per active slot.
__global__ void k_slot_tick(double* t, double* beta, int* k, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t[s] * t[s]));
  const double t2 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t1 * t1));
  t[s] = t1;
  beta[s] = (t1 - 1.0) / t2;
  k[s] += 1;
}

__global__ void k_slot_init(Slots sl, int slot, double invL, double lamL) {
  sl.t[slot] = 1.0;
  sl.beta[slot] = 0.0;  // (t_1 - 1) / t_2 with t_1 = 1
  sl.invL[slot] = invL;
  sl.lamL[slot] = lamL;
  sl.r2[slot] = 0.0;
  sl.k[slot] = 0;
}

__global__ void k_slot_copy(Slots sl, int dst, int src) {
  sl.t[dst] = sl.t[src];
  sl.beta[dst] = sl.beta[src];
  sl.invL[dst] = sl.invL[src];
  sl.lamL[dst] = sl.lamL[src];
  sl.r2[dst] = sl.r2[src];
  sl.k[dst] = sl.k[src];
}

size_t vol_bytes(const Layout& L) { return (size_t)L.nz * L.ny * L.nx * L.rsize; }
size_t dat_bytes(const Layout& L) { return (size_t)L.nt * L.my * L.mx * L.rsize; }

cudaError_t slot_step(pat_plan* pp, int n, cudaStream_t s) {
  Plan& p = pp->p;
  Slots& sl = pp->x.slots;
  const Layout& L = p.L;
  cudaError_t e = gradient_dev(p, p.vol_a, p.dat_b, p.vol_c, n, s, nullptr, n, sl.r2);
  if (e != cudaSuccess) return e;
  const int64_t vol = (int64_t)L.nz * L.ny * L.nx, tot = vol * n;
  int64_t g = (tot + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (L.fp64)
    e = launch_pdl(k_slot_update<double>, dim3((unsigned)g), dim3(256), 0, s,
                   static_cast<double*>(p.vol_a), static_cast<double*>(p.vol_b),
                   static_cast<const double*>(p.vol_c), vol, tot, sl.invL, sl.lamL, sl.beta);
  else
    e = launch_pdl(k_slot_update<float>, dim3((unsigned)g), dim3(256), 0, s,
                   static_cast<float*>(p.vol_a), static_cast<float*>(p.vol_b),
                   static_cast<const float*>(p.vol_c), vol, tot, sl.invL, sl.lamL, sl.beta);
  if (e != cudaSuccess) return e;
  k_slot_tick<<<(n + 127) / 128, 128, 0, s>>>(sl.t, sl.beta, sl.k, n);
  return cudaGetLastError();
}

Graph* step_graph(pat_plan* pp, int n, int* rc) {
  Plan& p = pp->p;
  for (Graph* g = p.graphs; g; g = g->next)
    if (g->kind == 1 && g->batch == n) return g;
  cudaStream_t cs = pp->x.cap;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t e2 = slot_step(pp, n, cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (e2 != cudaSuccess) e = e2;
  }
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  if (e == cudaSuccess) e = instantiate_counted(graph, &exec, &kernels);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "capturing the slot step graph");
    return nullptr;
  }
  Graph* g = new (std::nothrow) Graph();
  if (!g) {
    cudaGraphExecDestroy(exec);
    *rc = fail(PAT_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  g->kind = 1;
  g->batch = n;
  g->kernels = kernels;
  g->exec = exec;
  g->next = p.graphs;
  p.graphs = g;
  return g;
}

int check_slot(pat_plan* plan, int slot) {
  if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
  if (plan->p.shard_world)
    return fail(PAT_ERR_ARG, "a frequency-shard plan runs only the pat_shard_* stages");
  if (slot < 0 || slot >= plan->p.L.max_batch) return fail(PAT_ERR_ARG, "slot out of range");
  return PAT_OK;
}

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" {

int pat_slot_load(pat_plan* plan, int slot, const void* y, double lambda, double L,
                  pat_stream stream) {
  try {
    int rc = check_slot(plan, slot);
    if (rc != PAT_OK) return rc;
    if (!y) return fail(PAT_ERR_ARG, "y is NULL");
    if (!(L > 0) || !(lambda >= 0)) return fail(PAT_ERR_ARG, "need L > 0 and lambda >= 0");
    Plan& p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = vol_bytes(p.L), db = dat_bytes(p.L);
    char* dat = static_cast<char*>(p.dat_b) + slot * db;
    PAT_CUDA(cudaMemcpyAsync(dat, y, db, cudaMemcpyDefault, s));
    PAT_CUDA(cudaMemsetAsync(static_cast<char*>(p.vol_a) + slot * vb, 0, vb, s));
    PAT_CUDA(cudaMemsetAsync(static_cast<char*>(p.vol_b) + slot * vb, 0, vb, s));
    k_slot_init<<<1, 1, 0, s>>>(plan->x.slots, slot, 1.0 / L, lambda / L);
    PAT_CUDA(cudaGetLastError());
    if (!is_device_ptr(y)) PAT_CUDA(cudaStreamSynchronize(s));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_slot_move(pat_plan* plan, int dst, int src, pat_stream stream) {
  try {
    int rc = check_slot(plan, dst);
    if (rc == PAT_OK) rc = check_slot(plan, src);
    if (rc != PAT_OK) return rc;
    if (dst == src) return PAT_OK;
    Plan& p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = vol_bytes(p.L), db = dat_bytes(p.L);
    auto mv = [&](void* base, size_t sz) -> cudaError_t {
      char* b = static_cast<char*>(base);
      return cudaMemcpyAsync(b + dst * sz, b + src * sz, sz, cudaMemcpyDeviceToDevice, s);
    };
    PAT_CUDA(mv(p.dat_b, db));
    PAT_CUDA(mv(p.vol_a, vb));
    PAT_CUDA(mv(p.vol_b, vb));
    k_slot_copy<<<1, 1, 0, s>>>(plan->x.slots, dst, src);
    PAT_CUDA(cudaGetLastError());
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_slots_step(pat_plan* plan, int n, int* kernels, pat_stream stream) {
  try {
    if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
    if (plan->p.shard_world)
      return fail(PAT_ERR_ARG, "a frequency-shard plan runs only the pat_shard_* stages");
    if (n < 0 || n > plan->p.L.max_batch) return fail(PAT_ERR_ARG, "n must be in [0, max_batch]");
    if (kernels) *kernels = 0;
    if (n == 0) return PAT_OK;
    int rc = PAT_OK;
    Graph* g = step_graph(plan, n, &rc);
    if (!g) return rc;
    PAT_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    if (kernels) *kernels = g->kernels;
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_slot_read(pat_plan* plan, int slot, void* x, double* resid2, pat_stream stream) {
  try {
    int rc = check_slot(plan, slot);
    if (rc != PAT_OK) return rc;
    Plan& p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = vol_bytes(p.L);
    if (x)
      PAT_CUDA(cudaMemcpyAsync(x, static_cast<char*>(p.vol_b) + slot * vb, vb, cudaMemcpyDefault, s));
    if (resid2)
      PAT_CUDA(cudaMemcpyAsync(resid2, plan->x.slots.r2 + slot, sizeof(double),
                               cudaMemcpyDeviceToHost, s));
    if (resid2 || (x && !is_device_ptr(x))) PAT_CUDA(cudaStreamSynchronize(s));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

}  // extern "C"
