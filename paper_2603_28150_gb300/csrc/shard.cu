// Frequency-sharded operator (the multi-GPU split of Sec. 3.2's three stages):
// stage ii (Eq. 16 term (ii)) is independent per frequency bin, so `world`
// ranks each keep an equal range of the table's rows (the D4 representatives
// of a folded library, else bins) and contract only those; stages i and iii
// are split by slices (depths or time samples). Between them an all-to-all
// moves the slice spectra: rank r's stage i writes, for each of its slices,
// every bin straight into the slot of the rank that owns it in a send buffer
// [world][slices of r][W]; after the exchange rank r holds [all slices][W]
// (its bins of every slice), contracts, and the reverse exchange hands each
// rank the spectra of its own output slices. The slot maps are the only new
// piece: the FFT kernels already write and read spectra through a bin -> slot
// map, and the contraction kernels run unchanged on the shard's rows.
#include <algorithm>
#include <vector>

#include "pat_internal.h"

namespace pat {
namespace {

// FISTA update of Eq. 14-15 on plain arrays (a distributed solve keeps its
// iterates sliced by depth on every rank): x = max(y - g invL - lamL, 0),
// y <- x + beta (x - xprev), xprev <- x.
__global__ void k_fista_step(float* __restrict__ y, float* __restrict__ xprev,
                             const float* __restrict__ g, int64_t n, float invL, float lamL,
                             float beta) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float x = y[i] - g[i] * invL - lamL;
    x = x > 0.f ? x : 0.f;
    y[i] = x + beta * (x - xprev[i]);
    xprev[i] = x;
  }
}

// y = a x + b y on n floats.
__global__ void k_axpby(float* __restrict__ y, const float* __restrict__ x, int64_t n, float a,
                        float b) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

struct Part {
  bool fold;
  int64_t rows_total, Wr, W, row0, rows;
  int nz_local, nt_local;
};

int partition(const pat_geometry* g, int fold, int rank, int world, Part* pt,
              std::vector<int>* members, std::vector<int>* rep) {
  if (!g) return fail(PAT_ERR_ARG, "geometry is NULL");
  if (world < 1 || rank < 0 || rank >= world) return fail(PAT_ERR_ARG, "need 0 <= rank < world");
  if (g->nz % world || g->nt % world)
    return fail(PAT_ERR_UNSUPPORTED, "shards split nz and nt into equal slices: world must divide both");
  if (fold && g->px != g->py) return fail(PAT_ERR_ARG, "a folded table needs px == py");
  const int64_t K = (int64_t)(g->px / 2 + 1) * g->py;
  pt->fold = fold != 0;
  if (pt->fold) {
    std::vector<int> slot;
    fold_enumerate(g->px, *members, *rep, slot);
    pt->rows_total = (int64_t)members->size() / 4;
  } else {
    pt->rows_total = K;
  }
  const int64_t per = (pt->rows_total + world - 1) / world;
  pt->Wr = (per + 31) / 32 * 32;  // table rows live in blocks of 32
  pt->W = (pt->fold ? 4 : 1) * pt->Wr;
  pt->row0 = std::min<int64_t>(pt->rows_total, (int64_t)rank * pt->Wr);
  pt->rows = std::min<int64_t>(pt->rows_total - pt->row0, pt->Wr);
  pt->nz_local = g->nz / world;
  pt->nt_local = g->nt / world;
  return PAT_OK;
}

// Owner rank and slot of every bin, as positions in an exchange buffer of
// `slices` slices per rank.
void bin_positions(const Part& pt, int64_t K, const std::vector<int>& rep, int slices,
                   int32_t* map) {
  for (int64_t k = 0; k < K; ++k) {
    int64_t q, off;
    if (pt.fold) {
      const int64_t u = rep[k];
      q = u / pt.Wr;
      // the slot of bin k among its representative's members
      off = 4 * (u - q * pt.Wr);
    } else {
      q = k / pt.Wr;
      off = k - q * pt.Wr;
    }
    map[k] = (int32_t)(q * slices * pt.W + off);
  }
}

void fill_maps(const Part& pt, int64_t K, const std::vector<int>& members,
               const std::vector<int>& rep, int32_t* zmap, int32_t* tmap, int32_t* mem_local) {
  if (zmap) bin_positions(pt, K, rep, pt.nz_local, zmap);
  if (tmap) bin_positions(pt, K, rep, pt.nt_local, tmap);
  if (pt.fold) {
    // member i of a representative sits in slot 4 (u - row0 of its owner) + i
    for (int64_t u = 0; u < pt.rows_total; ++u)
      for (int i = 0; i < 4; ++i) {
        const int k = members[4 * u + i];
        if (k < 0) continue;
        if (zmap) zmap[k] += i;
        if (tmap) tmap[k] += i;
      }
    if (mem_local)
      for (int64_t j = 0; j < pt.Wr; ++j)
        for (int i = 0; i < 4; ++i) {
          const int64_t u = pt.row0 + j;
          mem_local[4 * j + i] = (j < pt.rows && members[4 * u + i] >= 0) ? (int32_t)(4 * j + i) : -1;
        }
  }
}

int check_shard(pat_plan* plan) {
  if (!plan) return fail(PAT_ERR_ARG, "plan is NULL");
  if (!plan->p.shard_world) return fail(PAT_ERR_ARG, "not a frequency-shard plan");
  return PAT_OK;
}

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" {

int pat_shard_layout(const pat_geometry* g, int fold, int rank, int world, pat_shard_info* info,
                     int32_t* zmap, int32_t* tmap, int32_t* members_local) {
  try {
    if (!info) return fail(PAT_ERR_ARG, "info is NULL");
    Part pt;
    std::vector<int> members, rep;
    int rc = partition(g, fold, rank, world, &pt, &members, &rep);
    if (rc != PAT_OK) return rc;
    const int64_t K = (int64_t)(g->px / 2 + 1) * g->py;
    fill_maps(pt, K, members, rep, zmap, tmap, members_local);
    pat_shard_info v{};
    v.world = world;
    v.rank = rank;
    v.nz_local = pt.nz_local;
    v.nt_local = pt.nt_local;
    v.folded = pt.fold ? 1 : 0;
    v.rows_total = pt.rows_total;
    v.rows_per_rank = pt.Wr;
    v.row0 = pt.row0;
    v.rows = pt.rows;
    v.slot_width = pt.W;
    v.bins = K;
    *info = v;
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_OOM, "host allocation failed");
  }
}

int pat_plan_create_kspace_shard(const pat_geometry* g, const pat_medium* m, int rank, int world,
                                 pat_stream stream, pat_plan** out) {
  try {
    if (!out) return fail(PAT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !m) return fail(PAT_ERR_ARG, "geometry or medium is NULL");
    if (g->flags & (PAT_FLAG_FP64 | PAT_FLAG_BF16_SPLIT))
      return fail(PAT_ERR_UNSUPPORTED, "frequency shards are single precision, CUDA-core");
    if (g->max_batch != 1) return fail(PAT_ERR_UNSUPPORTED, "frequency shards take max_batch = 1");
    if (!(m->c > 0 && m->dx > 0 && m->dy > 0 && m->dz > 0 && m->dt > 0))
      return fail(PAT_ERR_ARG, "medium: c, dx, dy, dz, dt must be > 0");
    if (m->z0 < 0 || m->mz < 2 || (m->mz & (m->mz - 1)) || m->mz <= m->z0 + g->nz)
      return fail(PAT_ERR_ARG, "medium: mz must be a power of two > z0 + nz, z0 >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    // the partition first: argument errors need no device
    const bool fold = (g->flags & (PAT_FLAG_FORCE_COMPLEX | PAT_FLAG_NO_FOLD)) == 0 &&
                      g->px == g->py && m->dx == m->dy;
    Part pt;
    std::vector<int> members, rep;
    int rc = partition(g, fold ? 1 : 0, rank, world, &pt, &members, &rep);
    if (rc != PAT_OK) return rc;
    pat_plan* pp = nullptr;
    rc = plan_create_common(g, out, &pp, std::max<int64_t>(pt.nz_local, pt.nt_local));
    if (rc != PAT_OK) return rc;
    Plan& p = pp->p;
    Layout& L = p.L;
    set_representation(L, (g->flags & PAT_FLAG_FORCE_COMPLEX) == 0);
    if (kspace_folds(L, *m, (g->flags & PAT_FLAG_NO_FOLD) == 0) != fold)
      rc = fail(PAT_ERR_CUDA, "internal: shard folding decision differs from the plan's");
    std::vector<int32_t> zmap((size_t)L.K), tmap((size_t)L.K), mloc;
    if (rc == PAT_OK) {
      if (fold) mloc.resize((size_t)pt.Wr * 4);
      fill_maps(pt, L.K, members, rep, zmap.data(), tmap.data(), fold ? mloc.data() : nullptr);
      // the table of this shard: its rows only, in the plan's blocked layout;
      // folded, the representatives of one radius among this shard's rows
      // share a stored row as in an unsharded plan (the contraction's blocks
      // then address the exchange slots through their block map)
      set_representation(L, L.real, fold);
      std::vector<int> bins;
      FoldBlocks fb;
      if (fold && pt.rows == 0) {  // no rows: an unread table of one block per chunk
        L.U = 0;
        L.Upad = pt.Wr;
        L.nub = L.nrb = L.nch = pt.Wr / 32;
      } else if (fold) {
        L.U = pt.rows;
        L.Upad = pt.Wr;
        L.nub = pt.Wr / 32;
        std::vector<int> local((size_t)pt.rows * 4);
        for (int64_t j = 0; j < 4 * pt.rows; ++j) local[j] = members[4 * pt.row0 + j];
        fold_blocks(g->px, local, pt.rows, (g->flags & PAT_FLAG_NO_RADIAL) == 0, fb);
        L.nrb = fb.nrb;
        L.nch = fb.nch;
        L.radial = fb.nch != fb.nrb;
        bins.resize(fb.row_rep.size());
        for (size_t r = 0; r < bins.size(); ++r) bins[r] = local[4 * (size_t)std::max(fb.row_rep[r], 0)];
        if (L.radial) {  // block slot -> exchange slots of its representative
          std::vector<int32_t> rbm(fb.rb_rep.size() * 4, -1);
          for (size_t v = 0; v < fb.rb_rep.size(); ++v)
            if (fb.rb_rep[v] >= 0)
              for (int i = 0; i < 4; ++i) rbm[4 * v + i] = mloc[4 * (size_t)fb.rb_rep[v] + i];
          mloc.swap(rbm);
        }
      } else {
        bins.resize((size_t)pt.rows);
        for (int64_t j = 0; j < pt.rows; ++j) bins[j] = (int)(pt.row0 + j);
      }
      const int64_t blocks = fold ? L.nch : pt.Wr / 32;
      L.table_bytes = (size_t)blocks * L.nt * L.nzg * 32 * 16;
      p.shard_world = world;
      p.shard_rank = rank;
      p.shard_row0 = pt.row0;
      p.shard_rows = pt.rows;
      p.shard_Wr = pt.Wr;
      p.shard_W = pt.W;
      cudaError_t e = dev_alloc(&p.shard_zmap, zmap.size() * sizeof(int32_t));
      if (e == cudaSuccess) e = dev_alloc(&p.shard_tmap, tmap.size() * sizeof(int32_t));
      if (e == cudaSuccess && fold) e = dev_alloc(&p.shard_members, mloc.size() * sizeof(int32_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(p.shard_zmap, zmap.data(), zmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(p.shard_tmap, tmap.data(), tmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && fold)
        e = cudaMemcpy(p.shard_members, mloc.data(), mloc.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
      if (e == cudaSuccess && fold && L.radial) e = dev_alloc(&p.rb_chunk, fb.rb_chunk.size() * sizeof(int));
      if (e == cudaSuccess && fold && L.radial)
        e = cudaMemcpy(p.rb_chunk, fb.rb_chunk.data(), fb.rb_chunk.size() * sizeof(int),
                       cudaMemcpyHostToDevice);
      if (e != cudaSuccess) rc = cuda_fail(e, "uploading the shard maps");
      if (rc == PAT_OK) rc = kspace_generate(p, *m, bins, s);
    }
    if (rc != PAT_OK) {
      plan_free(pp);
      return rc;
    }
    *out = pp;
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_OOM, "host allocation failed");
  }
}

int pat_plan_shard_info(const pat_plan* plan, pat_shard_info* info) {
  if (!plan || !info) return fail(PAT_ERR_ARG, "plan or info is NULL");
  const Plan& p = plan->p;
  if (!p.shard_world) return fail(PAT_ERR_ARG, "not a frequency-shard plan");
  const int64_t h = p.L.px / 2;
  pat_shard_info v{};
  v.world = p.shard_world;
  v.rank = p.shard_rank;
  v.nz_local = p.L.nz / p.shard_world;
  v.nt_local = p.L.nt / p.shard_world;
  v.folded = p.L.fold ? 1 : 0;
  // representatives of the half spectrum when folded, else bins
  v.rows_total = p.L.fold ? (h + 1) * (h + 2) / 2 : p.L.K;
  v.rows_per_rank = p.shard_Wr;
  v.row0 = p.shard_row0;
  v.rows = p.shard_rows;
  v.slot_width = p.shard_W;
  v.bins = p.L.K;
  *info = v;
  return PAT_OK;
}

int pat_shard_spectrum(pat_plan* plan, int side, const float* in, void* send, pat_stream stream) {
  try {
    int rc = check_shard(plan);
    if (rc != PAT_OK) return rc;
    if (side != 0 && side != 1) return fail(PAT_ERR_ARG, "side must be 0 (depths) or 1 (time samples)");
    if (!in || !send) return fail(PAT_ERR_ARG, "in or send is NULL");
    if (!is_device_ptr(in) || !is_device_ptr(send)) return fail(PAT_ERR_ARG, "device arrays required");
    const Plan& p = plan->p;
    const Layout& L = p.L;
    const int n = (side ? L.nt : L.nz) / p.shard_world;
    PAT_CUDA(launch_spectrum(p, in, (int64_t)L.ny * L.nx, L.nx, L.ny, send, p.shard_W, n,
                             (cudaStream_t)stream, no_sampling(), side ? p.shard_tmap : p.shard_zmap));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_shard_contract(pat_plan* plan, int adjoint, const void* in, void* out, pat_stream stream) {
  try {
    int rc = check_shard(plan);
    if (rc != PAT_OK) return rc;
    if (!in || !out) return fail(PAT_ERR_ARG, "in or out is NULL");
    if (!is_device_ptr(in) || !is_device_ptr(out)) return fail(PAT_ERR_ARG, "device arrays required");
    const Plan& p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    if (p.shard_rows == 0) return PAT_OK;  // no rows: nobody reads this rank's slots
    // the contraction kernels on this shard's rows: a view of the plan whose
    // row count and row stride are the shard's
    Plan v = p;
    v.tc_fwd = v.tc_adj = nullptr;
    v.tc_min_batch = 0;
    v.L.Kpad = p.shard_W;
    if (p.L.fold) {
      // block slots address this shard's exchange slots; with radial sharing
      // the blocks of a radius group read one chunk (else block j reads chunk j)
      v.rb_members = p.shard_members;
      v.rb_chunk = p.L.radial ? p.rb_chunk : nullptr;
    } else {
      v.L.K = p.shard_rows;
      v.L.nkb = p.shard_Wr / 32;
    }
    PAT_CUDA(adjoint ? launch_contract_adj(v, in, out, 1, s) : launch_contract_fwd(v, in, out, 1, s));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_shard_image(pat_plan* plan, int side, const void* recv, float* out, const float* sub,
                    double* r2, pat_stream stream) {
  try {
    int rc = check_shard(plan);
    if (rc != PAT_OK) return rc;
    if (side != 0 && side != 1) return fail(PAT_ERR_ARG, "side must be 0 (depths) or 1 (time samples)");
    if (!recv || !out) return fail(PAT_ERR_ARG, "recv or out is NULL");
    if (!is_device_ptr(recv) || !is_device_ptr(out) || (sub && !is_device_ptr(sub)))
      return fail(PAT_ERR_ARG, "device arrays required");
    if (r2 && !sub) return fail(PAT_ERR_ARG, "r2 needs sub");
    const Plan& p = plan->p;
    const Layout& L = p.L;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (side ? L.nt : L.nz) / p.shard_world;
    double* dsum = r2 ? plan->x.res + 3 : nullptr;
    PAT_CUDA(launch_image(p, recv, p.shard_W, out, (int64_t)L.ny * L.nx, n, sub, dsum, s, 0, nullptr,
                          no_sampling(), side ? p.shard_tmap : p.shard_zmap));
    if (r2) {
      PAT_CUDA(cudaMemcpyAsync(r2, dsum, sizeof(double), cudaMemcpyDeviceToHost, s));
      PAT_CUDA(cudaStreamSynchronize(s));
    }
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_fista_step(float* y, float* xprev, const float* grad, int64_t n, double invL, double lamL,
                   double beta, pat_stream stream) {
  try {
    if (n < 0 || (n > 0 && (!y || !xprev || !grad))) return fail(PAT_ERR_ARG, "bad arguments");
    if (n == 0) return PAT_OK;
    if (!is_device_ptr(y) || !is_device_ptr(xprev) || !is_device_ptr(grad))
      return fail(PAT_ERR_ARG, "device arrays required");
    if (!(invL > 0) || !(lamL >= 0)) return fail(PAT_ERR_ARG, "need invL > 0 and lamL >= 0");
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    PAT_CUDA(launch_pdl(k_fista_step, dim3((unsigned)blocks), dim3(256), 0, (cudaStream_t)stream, y,
                        xprev, grad, n, (float)invL, (float)lamL, (float)beta));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

int pat_axpby(float* y, const float* x, int64_t n, double a, double b, pat_stream stream) {
  try {
    if (n < 0 || (n > 0 && (!y || !x))) return fail(PAT_ERR_ARG, "bad arguments");
    if (n == 0) return PAT_OK;
    if (!is_device_ptr(y) || !is_device_ptr(x)) return fail(PAT_ERR_ARG, "device arrays required");
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    PAT_CUDA(launch_pdl(k_axpby, dim3((unsigned)blocks), dim3(256), 0, (cudaStream_t)stream, y, x,
                        n, (float)a, (float)b));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}

}  // extern "C"
