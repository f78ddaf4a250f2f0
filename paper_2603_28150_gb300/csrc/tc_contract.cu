// Batched depth contraction on the tcgen05 tensor cores (Sec. 3.2, Eq. 16
// term (ii)) for 16 volumes sharing one real (even-kernel) table:
//   forward  Y_k (nt x 2B) = H_k (nt x nz) X_k (nz x 2B)            (Eq. 7)
//   adjoint  Z_k (nz x 2B) = H_k^T (nz x nt) D_k (nt x 2B)          (Eq. 11)
// per frequency bin k, with the 2B columns = real and imaginary parts of the
// B = 16 volumes. Operands are split into BF16 hi + lo (h = hi + lo to ~2^-16
// relative) and the product is hi.hi + hi.lo + lo.hi with FP32 accumulation in
// tensor memory (the dropped lo.lo term is ~2^-16 of the others).
//
// Layout: the split table is stored per bin as 32 KB tiles of 128 x 128 BF16
// in the no-swizzle K-major core-matrix layout (8 rows x 16 B per core
// matrix; cores adjacent along K are 128 B apart, along M/N 2048 B apart), one
// copy per direction (forward: rows t, K = z; adjoint: rows z, K = t chunks),
// so each tile is one contiguous bulk copy. The X / D operand of a bin is
// converted to the same layout in shared memory by all threads.
//
// Per CTA (persistent, one per SM, 128 threads): groups of G bins; thread 0
// streams the group's table tiles through an S-slot mbarrier pipeline
// (cp.async.bulk), issues the MMAs (M=128, N=32, K=16) and commits them to
// the slot's "empty" barrier; after a group all four warps read the
// accumulators with tcgen05.ld and write Y / Z (G consecutive bins per row).
// Every wait is bounded: on timeout the kernel records an error, drains its
// own copies, frees tensor memory and returns.
//
// D4-folded plans (k_tc_fold) keep one tile set per representative {|kx|,
// |ky|} (a quarter of the bytes) and put its up to 4 bins side by side in the
// MMA's N dimension (N = 4 x 32); their spectra use the representative-slot
// layout (a representative's 4 bins in one 32-byte sector of every row), so
// a representative's operand chunk is a 3D box (32 bytes x 128 rows x 16
// volumes) that one tensor copy moves.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "pat_internal.h"

namespace pat {
namespace tc {

constexpr int kThreads = 128;
constexpr int kVB = 16;                  // volumes per pass
constexpr int kN = 2 * kVB;              // MMA N: re and im of each volume
constexpr int kTile = 128;               // M rows and K columns per table tile
constexpr int kTileBytes = kTile * kTile * 2;  // 32 KB of BF16
constexpr int kLBO = 128;                // bytes between K-adjacent core matrices
constexpr int kSBO = (kTile / 8) * 128;  // bytes between M/N-adjacent core matrices (2048)
constexpr int kBBytes = kN * kTile * 2;  // one 32 x 128 B-operand chunk (8 KB)
// Teardown drains (copies and MMAs still in flight after an abort) wait at
// most this long in total, measured on the global timer.
constexpr uint64_t kDrainNs = 2000000000ull;

// -------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded pipeline wait for the phase with the given parity: at most `limit`
// tests (mbarrier.try_wait itself suspends the thread for a bounded time, so
// the loop polls without sleeping); false on timeout. limit = 0 gives up at
// once (the plan's wait limit set to 0 exercises the abort path).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Teardown wait: until the phase completes or the global timer passes
// `deadline` (shared by all drain waits of a thread, so once it has passed the
// remaining drains return at once).
__device__ __forceinline__ bool drain_wait(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  while (!mbar_test(bar, parity))
    if (global_ns() > deadline) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: no swizzle, K-major core matrices.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;                // start address
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;  // leading (K) byte offset
  d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;  // stride (M/N) byte offset
  d |= 1ull << 46;                             // descriptor version for tcgen05
  return d;                                    // base offset 0, layout type 0 (no swizzle)
}
// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) inside a no-swizzle K-major tile.
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// hi = bf16(v), lo = bf16(v - hi), packed pairs for 8 consecutive K.
__device__ __forceinline__ void split8(const float* v, uint4* hi, uint4* lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * i]), h1 = __float2bfloat16_rn(v[2 * i + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(h1));
    h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  *hi = make_uint4(h[0], h[1], h[2], h[3]);
  *lo = make_uint4(l[0], l[1], l[2], l[3]);
}

struct Params {
  const unsigned char* table;  // split tiles of this direction
  const float2* in;            // X [b][nz][Kpad] (fwd) or D [b][nt][Kpad] (adj)
  float2* out;                 // Y [b][nt][Kpad] (fwd) or Z [b][nz][Kpad] (adj)
  int64_t K, Kpad;
  int nz, nt, batch;
  int rows_out;      // nt (fwd) or nz (adj)
  int rows_in;       // nz (fwd) or nt (adj)
  int mtiles;        // output row tiles: nt/128 (fwd) or 1 (adj)
  int kchunks;       // K chunks of 128: 1 (fwd) or nt/128 (adj)
  int* err;          // set to 1 on a timed-out wait
  uint32_t spin;     // pipeline wait limit (tests per wait)
};

// G bins per group, S pipeline slots.
template <int G, int S>
__global__ void __launch_bounds__(kThreads, 1) k_tc_contract(Params p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // [S table slots][G * kchunks * 2 B chunks][barriers]
  unsigned char* slots = smem;
  unsigned char* bops = smem + (size_t)S * kTileBytes;
  const int kc_n = p.kchunks;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bops + (size_t)G * kc_n * 2 * kBBytes);
  uint64_t* full = bars;          // [S]
  uint64_t* empty = bars + S;     // [S]
  uint64_t* accb = bars + 2 * S;  // [1] accumulators of a group complete
  uint64_t* drainb = accb + 1;    // [1] used only when aborting
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(bars + 2 * S + 2);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_base_s + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ngroups = (p.K + G - 1) / G;
  const int tiles_per_bin = p.mtiles * kc_n * 2;
  const int tiles_per_group = G * tiles_per_bin;
  // this CTA's groups: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int64_t my_groups =
      blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total_tiles = my_groups * tiles_per_group;
  constexpr int kCols = 512;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    mbar_init(drainb, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_base_s)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base_s;
  constexpr uint32_t idesc = idesc_bf16(kTile, kN);

  // global tile j of this CTA -> (group, bin in group, row tile, K chunk, part)
  auto tile_src = [&](int64_t j) -> const unsigned char* {
    const int64_t gi = j / tiles_per_group;
    const int r = (int)(j % tiles_per_group);
    const int g = r / tiles_per_bin, rr = r % tiles_per_bin;
    const int64_t k = (blockIdx.x + gi * gridDim.x) * G + g;
    const int64_t kk = k < p.K ? k : p.K - 1;  // ragged last group: any valid tile
    return p.table + ((kk * tiles_per_bin) + rr) * (int64_t)kTileBytes;
  };
  int64_t issued = 0, consumed = 0;
  auto issue = [&](int64_t j) -> bool {
    const int s = (int)(j % S);
    if (j >= S && !mbar_wait(&empty[s], (uint32_t)(((j / S) - 1) & 1), p.spin)) return false;
    mbar_arrive_expect_tx(&full[s], kTileBytes);
    bulk_g2s(slots + (size_t)s * kTileBytes, tile_src(j), kTileBytes, &full[s]);
    return true;
  };
  if (tid == 0) {
    while (issued < total_tiles && issued < S) {
      if (!issue(issued)) {
        *abort_s = 1;
        break;
      }
      ++issued;
    }
  }

  for (int64_t gi = 0; gi < my_groups && !*abort_s; ++gi) {
    const int64_t k0 = (blockIdx.x + gi * gridDim.x) * G;
    // ---- B operands of the group's bins: complex64 -> BF16 hi / lo, K-major
    // chunk (g, kc, part) at bops + ((g * kc_n + kc) * 2 + part) * kBBytes;
    // rows n = b (real part) and kVB + b (imaginary part), K = input row.
    const int octs = p.rows_in / 8;
    for (int it = tid; it < kVB * octs; it += kThreads) {
      const int b = it / octs, o = it % octs;
      float re[G][8], im[G][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int row = o * 8 + q;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          float2 v = make_float2(0.f, 0.f);
          if (b < p.batch && k0 + g < p.K)
            v = p.in[((int64_t)b * p.rows_in + row) * p.Kpad + k0 + g];
          re[g][q] = v.x;
          im[g][q] = v.y;
        }
      }
      const int kc = (o * 8) / kTile, kin = (o * 8) % kTile;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        unsigned char* base = bops + (size_t)((g * kc_n + kc) * 2) * kBBytes;
        uint4 h, l;
        split8(re[g], &h, &l);
        *reinterpret_cast<uint4*>(base + core_off(b, kin)) = h;
        *reinterpret_cast<uint4*>(base + kBBytes + core_off(b, kin)) = l;
        split8(im[g], &h, &l);
        *reinterpret_cast<uint4*>(base + core_off(kVB + b, kin)) = h;
        *reinterpret_cast<uint4*>(base + kBBytes + core_off(kVB + b, kin)) = l;
      }
    }
    fence_proxy_async();
    __syncthreads();

    // ---- MMAs of the group (thread 0), table tiles streamed through the slots
    if (tid == 0) {
      tc_fence_after();
      for (int r = 0; r < tiles_per_group; ++r) {
        const int64_t j = gi * tiles_per_group + r;
        const int s = (int)(j % S);
        if (!mbar_wait(&full[s], (uint32_t)((j / S) & 1), p.spin)) {
          *abort_s = 1;
          break;
        }
        tc_fence_after();
        const int g = r / tiles_per_bin, rr = r % tiles_per_bin;
        const int part = rr & 1, kc = (rr >> 1) % kc_n, mt = (rr >> 1) / kc_n;
        const unsigned char* a = slots + (size_t)s * kTileBytes;
        const unsigned char* bh = bops + (size_t)((g * kc_n + kc) * 2) * kBBytes;
        const unsigned char* bl = bh + kBBytes;
        const uint32_t d = tmem + (uint32_t)((g * p.mtiles + mt) * kN);
#pragma unroll
        for (int ks = 0; ks < kTile / 16; ++ks) {
          const uint32_t off = ks * 2 * kLBO;
          const uint64_t ad = smem_desc(a + off);
          // hi tile: hi.hi and hi.lo; lo tile: lo.hi
          const uint32_t first = (part == 0 && kc == 0 && ks == 0) ? 0u : 1u;
          mma_bf16(d, ad, smem_desc(bh + off), idesc, first);
          if (part == 0) mma_bf16(d, ad, smem_desc(bl + off), idesc, 1u);
        }
        mma_commit(&empty[s]);
        ++consumed;
        if (issued < total_tiles) {
          if (!issue(issued)) {
            *abort_s = 1;
            break;
          }
          ++issued;
        }
      }
      mma_commit(accb);
    }
    // ---- epilogue: accumulators -> Y / Z rows of this warp's TMEM lanes
    // warp-uniform, since tcgen05.ld below is a warp-collective instruction
    const bool ok = __all_sync(0xffffffffu, mbar_wait(accb, (uint32_t)(gi & 1), p.spin));
    if (!ok) *abort_s = 1;
    tc_fence_after();
    __syncwarp();
    if (ok) {
      for (int mt = 0; mt < p.mtiles; ++mt) {
        const int row = mt * kTile + warp * 32 + lane;
        float v[G][kN];
#pragma unroll
        for (int g = 0; g < G; ++g)
          tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((g * p.mtiles + mt) * kN),
                    v[g]);
        if (row < p.rows_out) {
          for (int b = 0; b < p.batch && b < kVB; ++b) {
            float2* o = p.out + ((int64_t)b * p.rows_out + row) * p.Kpad + k0;
#pragma unroll
            for (int g = 0; g < G; ++g)
              if (k0 + g < p.K) o[g] = make_float2(v[g][b], v[g][kVB + b]);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }

  // ---- teardown (also after a timeout): drain our copies, free tensor memory
  if (tid == 0 && *abort_s) {
    atomicExch(p.err, 1);
    const uint64_t deadline = global_ns() + kDrainNs;
    for (int64_t j = consumed; j < issued; ++j)
      drain_wait(&full[j % S], (uint32_t)((j / S) & 1), deadline);
    mma_commit(drainb);  // arrives once every MMA issued so far has completed
    drain_wait(drainb, 0, deadline);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
}

// ---- D4-folded tables: one tile set per representative, N = 4 bins x 32 -----
// Per representative u the MMA's B operand holds its (up to) 4 member bins:
// row n = m * 32 + h * 16 + b is the real (h = 0) or imaginary (h = 1) part of
// volume b at bin members[u][m], so one pass over u's tiles serves all 4 bins
// (the table is read once per representative instead of once per bin).
// Warp roles (192 threads): warp 0 streams the table tiles (cp.async.bulk,
// kFS-slot ring); warp 1 issues the MMAs (and, in the adjoint, stages each
// operand chunk by one 3D tensor copy as soon as the previous one has been
// read out); warps 2-5 convert the staged FP32 operand chunk into the BF16
// hi / lo B operand and drain the accumulators (two alternating TMEM buffers
// of 256 columns): the forward through the staging buffer and 3D tensor
// stores, the adjoint by direct stores spread over the next representative's
// chunks. Table streaming, conversion, MMAs and drains of consecutive
// representatives overlap.
//   forward: M = 128 time samples of tile mt, K = nz = 128, accumulator units
//            of two time tiles; one B chunk per representative;
//   adjoint: M = nz = 128 depths, K = 128-sample chunks kc of nt, one
//            accumulator per representative; one B chunk per kc.
constexpr int kFS = 3;                    // table slots
constexpr int kFThreads = 192;
constexpr int kFN = 128;                  // MMA N: 4 members x (re, im) x 16 volumes
constexpr int kFBBytes = kFN * kTile * 2;  // one part (hi or lo) of a B chunk: 32 KB
// staged FP32 operand chunk: 16 volumes x 128 rows x one representative's 4
// complex members (32 bytes)
constexpr int kStageBytes = kVB * kTile * 32;

struct FoldParams {
  const unsigned char* table;  // split tiles of this direction, per representative
  const int4* members;         // [U] bins of each representative (-1 = none)
  const float2* in;            // X [b][nz][srow] (fwd) or D [b][nt][srow] (adj), slot layout
  float2* out;                 // Y [b][nt][srow] (fwd) or Z [b][nz][srow] (adj), slot layout
  int64_t U, srow;
  int batch;
  int rows_in, rows_out;  // nz, nt (fwd) or nt, nz (adj)
  int R;                  // tile rows per representative: mtiles (fwd) or kchunks (adj)
  int* err;
  uint32_t spin;          // pipeline wait limit (tests per wait)
};

// Bounded pipeline wait (at most `limit` tests, see mbar_wait) that also gives
// up once another role has aborted; a wait that runs out sets the abort flag.
__device__ __forceinline__ bool fwait(uint64_t* bar, uint32_t parity, volatile int* abort_s,
                                      uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (*abort_s) return false;
  }
  *abort_s = 1;
  return false;
}
// Warp-uniform form: every lane polls, all lanes get the same answer.
__device__ __forceinline__ bool fwait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_s,
                                           uint32_t limit) {
  return __all_sync(0xffffffffu, fwait(bar, parity, abort_s, limit));
}
__device__ __forceinline__ int member(int4 v, int m) {
  return m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 3D tiled tensor copy shared -> global (volumes past the tensor's extent are
// not written), committed as a bulk group; x is a multiple of 8 floats.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// 3D tiled tensor copy global -> shared completing on `bar`; x (the innermost
// coordinate, in floats) is a multiple of 8, so it starts on a 32-byte boundary.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <bool ADJ>
__global__ void __launch_bounds__(kFThreads, 1)
    k_tc_fold(FoldParams p, const __grid_constant__ CUtensorMap tin,
              const __grid_constant__ CUtensorMap tout) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* slots = smem;                               // [kFS][32 KB]
  unsigned char* bbuf = smem + (size_t)kFS * kTileBytes;     // [hi 32 KB | lo 32 KB]
  unsigned char* stage = bbuf + 2 * (size_t)kFBBytes;        // in: [128 rows][16 b][8 floats]; out: [16 b][128 rows][8 floats]
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + kStageBytes);
  uint64_t* full = bars;             // [kFS] tile landed
  uint64_t* empty = bars + kFS;      // [kFS] tile consumed by the MMAs
  uint64_t* bready = bars + 2 * kFS;  // [1] B chunk written (128 arrivals)
  uint64_t* bfree = bready + 1;       // [1] B chunk consumed by the MMAs
  uint64_t* sfull = bfree + 1;        // [1] operand chunk staged by the tensor copy
  uint64_t* sfree = sfull + 1;        // [1] staged chunk read out (128 arrivals; adjoint)
  uint64_t* afull = sfree + 1;        // [2] accumulator buffer complete
  uint64_t* aempty = afull + 2;       // [2] accumulator buffer drained (128 arrivals)
  uint64_t* drainb = aempty + 2;      // [1] all MMAs done (teardown)
  uint64_t* gbar = drainb + 1;        // [1] barrier of the 4 gather warps (128 arrivals)
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(gbar + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_base_s + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nmine = blockIdx.x < p.U ? (p.U - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int R = p.R;
  // forward: accumulator units of two time tiles; adjoint: one per representative
  const int NA = ADJ ? 1 : (R + 1) / 2;
  const int NB = ADJ ? R : 1;  // B chunks per representative
  constexpr int kCols = 512;

  if (tid == 0) {
    for (int s = 0; s < kFS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(bready, 128);
    mbar_init(bfree, 1);
    mbar_init(sfull, 1);
    mbar_init(sfree, 128);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 128);
    }
    mbar_init(drainb, 1);
    mbar_init(gbar, 128);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_base_s)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base_s;
  int64_t issued = 0;  // table tiles copied (warp 0)
  int64_t staged = 0;  // operand chunks staged (warp 1)

  if (warp == 0) {
    // ---- producer: the tiles of this CTA's representatives, in MMA order
    const int64_t total = nmine * 2 * R;
    for (int64_t j = 0; j < total && !*abort_s; ++j) {
      const int s = (int)(j % kFS);
      if (j >= kFS &&
          !fwait_warp(&empty[s], (uint32_t)(((j / kFS) - 1) & 1), abort_s, p.spin))
        break;
      if (lane == 0) {
        const int64_t u = blockIdx.x + (j / (2 * R)) * gridDim.x;
        const int64_t tile = u * 2 * R + j % (2 * R);
        mbar_arrive_expect_tx(&full[s], kTileBytes);
        bulk_g2s(slots + (size_t)s * kTileBytes, p.table + tile * (int64_t)kTileBytes, kTileBytes,
                 &full[s]);
      }
      issued = j + 1;
      __syncwarp();
    }
  } else if (warp == 1) {
    // ---- MMA issuer (lane 0); tile j of representative i is (r, part) = (j / 2, j % 2).
    // It also stages the operand chunks: chunk c = (representative i, K chunk
    // kc), c = i * NB + kc, is one 3D tensor copy (8 floats x 128 rows x 16
    // volumes: the 32-byte member groups of one representative; volumes past
    // the batch read as zero) into the staging buffer, issued as soon as the
    // gather warps have read chunk c - 1 out of it (before they convert it).
    // The forward stages its one chunk per representative from the gather
    // warps instead (the staging buffer also carries its output tiles).
    constexpr uint32_t idesc = idesc_bf16(kTile, kFN);
    const int64_t nchunks = nmine * NB;
    auto stage_chunk = [&](int64_t c) {
      if (lane == 0) {
        const int64_t u = blockIdx.x + (c / NB) * gridDim.x;
        mbar_arrive_expect_tx(sfull, kStageBytes);
        tma_load_3d(stage, &tin, (int)(8 * u), 0, (int)(c % NB) * kTile, sfull);
      }
      staged = c + 1;
      __syncwarp();
    };
    if (ADJ && nchunks > 0) stage_chunk(0);
    int64_t j = 0;
    for (int64_t i = 0; i < nmine && !*abort_s; ++i) {
      bool ok = true;
      for (int r = 0; r < R && ok; ++r) {
        const int64_t c = ADJ ? i * NB + r : i;  // B chunk
        if (ADJ) {
          // chunk c read out of the staging buffer: stage chunk c + 1
          ok = fwait_warp(sfree, (uint32_t)(c & 1), abort_s, p.spin);
          if (ok && c + 1 < nchunks) stage_chunk(c + 1);
        }
        if (ok && (ADJ || r == 0)) ok = fwait_warp(bready, (uint32_t)(c & 1), abort_s, p.spin);
        const int64_t q = ADJ ? i : i * NA + r / 2;  // accumulator unit
        const bool unit_start = ADJ ? r == 0 : (r % 2 == 0);
        if (ok && unit_start && q >= 2)
          ok = fwait_warp(&aempty[q & 1], (uint32_t)(((q >> 1) - 1) & 1), abort_s, p.spin);
        if (!ok) break;
        tc_fence_after();
        const unsigned char* bh = bbuf;
        const unsigned char* bl = bh + kFBBytes;
        const uint32_t d = tmem + (uint32_t)((q & 1) * 256 + (ADJ ? 0 : (r % 2) * 128));
        for (int part = 0; part < 2 && ok; ++part, ++j) {
          const int s = (int)(j % kFS);
          ok = fwait_warp(&full[s], (uint32_t)((j / kFS) & 1), abort_s, p.spin);
          if (!ok) break;
          tc_fence_after();
          if (lane == 0) {
            const unsigned char* a = slots + (size_t)s * kTileBytes;
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks) {
              const uint32_t off = ks * 2 * kLBO;
              const uint64_t ad = smem_desc(a + off);
              // hi tile: hi.hi and hi.lo; lo tile: lo.hi
              const bool first = part == 0 && ks == 0 && (ADJ ? r == 0 : true);
              mma_bf16(d, ad, smem_desc(bh + off), idesc, first ? 0u : 1u);
              if (part == 0) mma_bf16(d, ad, smem_desc(bl + off), idesc, 1u);
            }
            mma_commit(&empty[s]);
          }
          __syncwarp();
        }
        if (!ok) break;
        const bool unit_end = ADJ ? r == R - 1 : (r % 2 == 1 || r == R - 1);
        if (lane == 0) {
          if (ADJ || r == R - 1) mma_commit(bfree);
          if (unit_end) mma_commit(&afull[q & 1]);
        }
        __syncwarp();
      }
    }
  } else {
    // ---- gather + split (B operand) and epilogue (accumulators -> Y / Z)
    const int ct = tid - 64;     // 0..127
    const int quarter = warp & 3;  // TMEM lanes 32 * quarter ... of this warp
    // Operands in the slot layout: row (b, r) of X / D holds the 4 members of
    // representative u at [4u, 4u + 4) of its srow complex values (32 bytes).
    auto gather = [&](int64_t i, int kc, int64_t c) -> bool {
      (void)kc;
      if (!fwait_warp(sfull, (uint32_t)(c & 1), abort_s, p.spin)) return false;
      tc_fence_after();
      const int64_t u = blockIdx.x + i * gridDim.x;
      const int4 mem = p.members[u];
      unsigned char* bh = bbuf;
      const float* sf = reinterpret_cast<const float*>(stage);
      // items (b, octet of rows): 16 x 16, two per thread; both read out of
      // the staging buffer first, so (adjoint) the next chunk's copy can start
      // while this one is converted
      float4 lo4s[2][8], hi4s[2][8];  // members (0, 1) and (2, 3) of 8 rows
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int it = ct + k * 128;
        const int b = it & 15, oct = it >> 4;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4* src =
              reinterpret_cast<const float4*>(sf + ((size_t)(oct * 8 + q) * kVB + b) * 8);
          lo4s[k][q] = src[0];
          hi4s[k][q] = src[1];
        }
      }
      if (ADJ) {
        fence_proxy_async();
        mbar_arrive(sfree);
      }
      // the B buffer is free once the MMAs of chunk c - 1 are done
      if (c >= 1 && !fwait_warp(bfree, (uint32_t)((c - 1) & 1), abort_s, p.spin)) return false;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int it = ct + k * 128;
        const int b = it & 15, oct = it >> 4;
        const float4* lo4 = lo4s[k];
        const float4* hi4 = hi4s[k];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const bool present = member(mem, m) >= 0;
          float re[8], im[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 w = m < 2 ? lo4[q] : hi4[q];
            re[q] = present ? ((m & 1) ? w.z : w.x) : 0.f;
            im[q] = present ? ((m & 1) ? w.w : w.y) : 0.f;
          }
          uint4 h, l;
          split8(re, &h, &l);
          *reinterpret_cast<uint4*>(bh + core_off(m * 32 + b, oct * 8)) = h;
          *reinterpret_cast<uint4*>(bh + kFBBytes + core_off(m * 32 + b, oct * 8)) = l;
          split8(im, &h, &l);
          *reinterpret_cast<uint4*>(bh + core_off(m * 32 + 16 + b, oct * 8)) = h;
          *reinterpret_cast<uint4*>(bh + kFBBytes + core_off(m * 32 + 16 + b, oct * 8)) = l;
        }
      }
      fence_proxy_async();  // B visible to the MMAs
      mbar_arrive(bready);
      return true;
    };
    // Adjoint drain of representative i in `parts` shares of the volumes:
    // share `part` stores volumes [part * 16 / parts, (part + 1) * 16 / parts).
    auto epilogue_adj = [&](int64_t i, int part, int parts) -> bool {
      if (part == 0 && !fwait_warp(&afull[i & 1], (uint32_t)((i >> 1) & 1), abort_s, p.spin))
        return false;
      tc_fence_after();
      const int64_t u = blockIdx.x + i * gridDim.x;
      const int row = quarter * 32 + lane;
      const int b0 = part * kVB / parts, b1 = (part + 1) * kVB / parts;
      float v[4][32];
      const uint32_t col = (uint32_t)((i & 1) * 256);
#pragma unroll
      for (int m = 0; m < 4; ++m)
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + col + (uint32_t)(m * 32), v[m]);
#pragma unroll
      for (int bb = 0; bb < kVB; ++bb) {
        if (bb < b0 || bb >= b1 || bb >= p.batch) continue;
        float4* o =
            reinterpret_cast<float4*>(p.out + ((int64_t)bb * p.rows_out + row) * p.srow + 4 * u);
        o[0] = make_float4(v[0][bb], v[0][16 + bb], v[1][bb], v[1][16 + bb]);
        o[1] = make_float4(v[2][bb], v[2][16 + bb], v[3][bb], v[3][16 + bb]);
      }
      if (part == parts - 1) {
        tc_fence_before();
        mbar_arrive(&aempty[i & 1]);
      }
      return true;
    };
    // ---- forward: the staging buffer alternates between the X chunk of the
    // next representative and the output tiles of the current one, which
    // leave by 3D tensor stores (one per 128-sample tile: 16 volumes x 128
    // rows x 32 bytes; volumes past the batch are not written).
    uint32_t gph = 0;  // phase of the gather-warp barrier
    auto gsync = [&]() -> bool {
      mbar_arrive(gbar);
      const bool ok = fwait_warp(gbar, gph & 1, abort_s, p.spin);
      ++gph;
      return ok;
    };
    int64_t fstaged = 0;  // forward X chunks staged (thread ct 0)
    auto stage_x = [&](int64_t i) {
      if (ct == 0) {
        const int64_t u = blockIdx.x + i * gridDim.x;
        mbar_arrive_expect_tx(sfull, kStageBytes);
        tma_load_3d(stage, &tin, (int)(8 * u), 0, 0, sfull);
        fstaged = i + 1;
      }
    };
    auto epilogue_fwd = [&](int64_t i, int a, int64_t q) -> bool {
      if (!fwait_warp(&afull[q & 1], (uint32_t)((q >> 1) & 1), abort_s, p.spin)) return false;
      tc_fence_after();
      const int64_t u = blockIdx.x + i * gridDim.x;
      const int nmt = min(2, R - 2 * a);
      const int r = quarter * 32 + lane;  // row of the 128-sample tile
      float* sf = reinterpret_cast<float*>(stage);
      for (int h = 0; h < nmt; ++h) {
        float v[4][32];
        const uint32_t col = (uint32_t)((q & 1) * 256 + h * 128);
#pragma unroll
        for (int m = 0; m < 4; ++m)
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + col + (uint32_t)(m * 32), v[m]);
        // the staging buffer is free (X read out, previous tile's store read)
        if (!gsync()) return false;
#pragma unroll
        for (int bb = 0; bb < kVB; ++bb) {
          float4* o = reinterpret_cast<float4*>(sf + ((size_t)bb * kTile + r) * 8);
          o[0] = make_float4(v[0][bb], v[0][16 + bb], v[1][bb], v[1][16 + bb]);
          o[1] = make_float4(v[2][bb], v[2][16 + bb], v[3][bb], v[3][16 + bb]);
        }
        fence_proxy_async();
        if (!gsync()) return false;
        if (ct == 0) {
          tma_store_3d(&tout, stage, (int)(8 * u), (2 * a + h) * kTile, 0);
          bulk_wait_read();
        }
      }
      tc_fence_before();
      mbar_arrive(&aempty[q & 1]);
      return true;
    };
    bool ok = true;
    if (!ADJ) {
      // X(0) staged, read out; X(1) staged; then per representative i: read
      // out X(i + 1), drain i through the staging buffer, stage X(i + 2)
      if (nmine > 0) {
        stage_x(0);
        ok = gather(0, 0, 0);
        if (ok && nmine > 1) {
          ok = gsync();
          if (ok) stage_x(1);
        }
      }
      for (int64_t i = 0; i < nmine && ok; ++i) {
        if (i + 1 < nmine) ok = gather(i + 1, 0, i + 1);
        for (int a = 0; a < NA && ok; ++a) ok = epilogue_fwd(i, a, i * NA + a);
        // thread ct 0 waited for its last store's read; the others wrote the
        // tile before the barrier that preceded it
        if (ok && i + 2 < nmine) stage_x(i + 2);
      }
      // after an abort: the staging copy still in flight lands before the
      // shared memory is released, and every store has read its tile
      if (ct == 0) {
        if (*abort_s && fstaged > 0)
          drain_wait(sfull, (uint32_t)((fstaged - 1) & 1), global_ns() + kDrainNs);
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      }
    } else {
      // the drain of representative i - 1 is spread over the K chunks of i
      // (a share of the volumes after each gather), filling the waits for the
      // staged chunks
      for (int64_t i = 0; i < nmine && ok; ++i) {
        for (int kc = 0; kc < NB && ok; ++kc) {
          ok = gather(i, kc, i * NB + kc);
          if (ok && i >= 1) ok = epilogue_adj(i - 1, kc, NB);
        }
      }
      for (int part = 0; part < NB && ok && nmine > 0; ++part)
        ok = epilogue_adj(nmine - 1, part, NB);
    }
  }

  // ---- teardown (also after a timeout): drain our copies, free tensor memory
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_s) {
    atomicExch(p.err, 1);
    // every copy issued lands before the shared memory is released
    const uint64_t deadline = global_ns() + kDrainNs;
    for (int64_t j = issued - kFS < 0 ? 0 : issued - kFS; j < issued; ++j)
      drain_wait(&full[j % kFS], (uint32_t)((j / kFS) & 1), deadline);
  }
  if (warp == 1 && lane == 0 && *abort_s) {
    const uint64_t deadline = global_ns() + kDrainNs;
    mma_commit(drainb);  // arrives once every MMA issued so far has completed
    drain_wait(drainb, 0, deadline);
    // the last staging copy issued lands before the shared memory is released
    if (staged > 0) drain_wait(sfull, (uint32_t)((staged - 1) & 1), deadline);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
}

size_t fold_smem() {
  return (size_t)kFS * kTileBytes + 2 * (size_t)kFBBytes + kStageBytes + 8 * (2 * kFS + 10) + 16;
}

template <int G, int S>
size_t smem_for(int kchunks) {
  return (size_t)S * kTileBytes + (size_t)G * kchunks * 2 * kBBytes + 8 * (2 * S + 2) + 16;
}

// Forward-direction tile of bin k, row tile mt (t rows), part, from the real
// blocked FP32 table (row rep[k] of the stored table, or row k when rep is
// NULL); adjoint tile of bin k, K chunk kc (t columns), part.
__global__ void k_split_tables(const float* __restrict__ table, const int* __restrict__ rep,
                               int nz, int nt, int nzg, int64_t K,
                               unsigned char* __restrict__ fwd, unsigned char* __restrict__ adj) {
  const int64_t n = K * nt * nz;
  const int mtiles = nt / kTile;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(i % nz);
    const int t = (int)((i / nz) % nt);
    const int64_t k = i / ((int64_t)nz * nt);
    const int64_t row = rep ? rep[k] : k;  // folded tables: the bin's representative row
    const int64_t kb = row >> 5, l = row & 31;
    const float h = table[(((kb * nt + t) * nzg + z / 4) * 32 + l) * 4 + z % 4];
    const __nv_bfloat16 hi = __float2bfloat16_rn(h);
    const __nv_bfloat16 lo = __float2bfloat16_rn(h - __bfloat162float(hi));
    // forward: tile (k, mt = t / 128), rows t % 128, K = z
    {
      const int64_t tb = (k * mtiles + t / kTile) * 2;
      const uint32_t off = core_off(t % kTile, z);
      *reinterpret_cast<__nv_bfloat16*>(fwd + tb * kTileBytes + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(fwd + (tb + 1) * kTileBytes + off) = lo;
    }
    // adjoint: tile (k, kc = t / 128), rows z, K = t % 128
    {
      const int64_t tb = (k * mtiles + t / kTile) * 2;
      const uint32_t off = core_off(z, t % kTile);
      *reinterpret_cast<__nv_bfloat16*>(adj + tb * kTileBytes + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(adj + (tb + 1) * kTileBytes + off) = lo;
    }
  }
}

}  // namespace tc

bool tc_supported(const Layout& L) {
  return !L.fp64 && L.real && L.nz == tc::kTile && L.nt % tc::kTile == 0 && L.nt <= 4 * tc::kTile;
}

// Folded plans keep one tile set per representative, the others one per bin.
size_t tc_table_bytes(const Layout& L) {
  const int64_t rows = L.fold ? L.U : L.K;
  return (size_t)rows * (L.nt / tc::kTile) * 2 * tc::kTileBytes;  // one direction
}

cudaError_t tc_build_tables(const Plan& p, void* fwd, void* adj, cudaStream_t s) {
  const Layout& L = p.L;
  // folded: tile set u is the stored row of representative u (row u, or
  // rep_row[u] with radial sharing)
  const int64_t rows = L.fold ? L.U : L.K;
  int64_t n = rows * L.nt * L.nz;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  tc::k_split_tables<<<(int)g, 256, 0, s>>>(static_cast<const float*>(p.table),
                                            L.fold ? p.rep_row : nullptr, L.nz,
                                            L.nt, L.nzg, rows, static_cast<unsigned char*>(fwd),
                                            static_cast<unsigned char*>(adj));
  return cudaGetLastError();
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of the operand (or result) spectra of one pass of up to 16 volumes in the
// representative-slot layout, seen as FP32 [nb][rows][2 srow]: a box of 8
// floats x 128 rows x 16 volumes is one representative's operand chunk
// (volumes past nb read as zero). With rows_outer the map's dimensions are
// ordered (x, volume, row), so the box lands in shared memory as
// [row][volume][8 floats] and the gather threads of one row octet read
// neighbouring 32-byte groups. The encoder comes from the driver at run
// time (the library does not link the driver API).
EncodeTiledFn load_encoder() {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<EncodeTiledFn>(f);
}

cudaError_t encode_operand_map(CUtensorMap* map, const void* base, int64_t srow, int rows,
                               int nb, bool rows_outer = false) {
  static const EncodeTiledFn encode = load_encoder();  // resolved once, thread-safe
  if (!encode) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {(cuuint64_t)(2 * srow), (cuuint64_t)rows, (cuuint64_t)nb};
  cuuint64_t strides[2] = {(cuuint64_t)(srow * 8), (cuuint64_t)(srow * 8 * rows)};
  cuuint32_t box[3] = {8, (cuuint32_t)tc::kTile, (cuuint32_t)tc::kVB};
  if (rows_outer) {
    dims[1] = (cuuint64_t)nb;
    dims[2] = (cuuint64_t)rows;
    strides[0] = (cuuint64_t)(srow * 8 * rows);
    strides[1] = (cuuint64_t)(srow * 8);
    box[1] = (cuuint32_t)tc::kVB;
    box[2] = (cuuint32_t)tc::kTile;
  }
  const cuuint32_t step[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims,
                            strides, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// Forward (adjoint = false) or adjoint contraction of `batch` volumes in
// passes of 16 through the tensor cores.
cudaError_t tc_contract(const Plan& p, const void* tables_fwd, const void* tables_adj,
                        const void* in, void* out, int batch, bool adjoint, int* err,
                        cudaStream_t s) {
  const Layout& L = p.L;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (L.fold) {
    const size_t smem = tc::fold_smem();
    auto fn = adjoint ? tc::k_tc_fold<true> : tc::k_tc_fold<false>;
    e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    const int rows_in = adjoint ? L.nt : L.nz, rows_out = adjoint ? L.nz : L.nt;
    for (int b0 = 0; b0 < batch; b0 += tc::kVB) {
      tc::FoldParams q;
      q.table = static_cast<const unsigned char*>(adjoint ? tables_adj : tables_fwd);
      q.members = reinterpret_cast<const int4*>(p.fold_members);
      q.in = static_cast<const float2*>(in) + (int64_t)b0 * rows_in * 4 * L.Upad;
      q.out = static_cast<float2*>(out) + (int64_t)b0 * rows_out * 4 * L.Upad;
      q.U = L.U;
      q.srow = 4 * L.Upad;
      q.batch = std::min(tc::kVB, batch - b0);
      q.rows_in = rows_in;
      q.rows_out = rows_out;
      q.R = L.nt / tc::kTile;
      q.err = err;
      q.spin = (uint32_t)p.tc_spin;
      CUtensorMap map_in, map_out;
      if ((e = encode_operand_map(&map_in, q.in, q.srow, rows_in, q.batch, true)) != cudaSuccess ||
          (e = encode_operand_map(&map_out, q.out, q.srow, rows_out, q.batch)) != cudaSuccess)
        return e;
      const int grid = (int)std::min<int64_t>(L.U, sms);
      fn<<<grid, tc::kFThreads, smem, s>>>(q, map_in, map_out);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int b0 = 0; b0 < batch; b0 += tc::kVB) {
    tc::Params q;
    q.K = L.K;
    q.Kpad = L.Kpad;
    q.nz = L.nz;
    q.nt = L.nt;
    q.batch = std::min(tc::kVB, batch - b0);
    q.err = err;
    q.spin = (uint32_t)p.tc_spin;
    if (!adjoint) {
      q.table = static_cast<const unsigned char*>(tables_fwd);
      q.in = static_cast<const float2*>(in) + (int64_t)b0 * L.nz * L.Kpad;
      q.out = static_cast<float2*>(out) + (int64_t)b0 * L.nt * L.Kpad;
      q.rows_out = L.nt;
      q.rows_in = L.nz;
      q.mtiles = L.nt / tc::kTile;
      q.kchunks = 1;
      constexpr int G = 4, S = 4;
      const size_t smem = tc::smem_for<G, S>(1);
      e = cudaFuncSetAttribute((const void*)tc::k_tc_contract<G, S>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const int64_t groups = (L.K + G - 1) / G;
      const int grid = (int)std::min<int64_t>(groups, sms);
      tc::k_tc_contract<G, S><<<grid, tc::kThreads, smem, s>>>(q);
    } else {
      q.table = static_cast<const unsigned char*>(tables_adj);
      q.in = static_cast<const float2*>(in) + (int64_t)b0 * L.nt * L.Kpad;
      q.out = static_cast<float2*>(out) + (int64_t)b0 * L.nz * L.Kpad;
      q.rows_out = L.nz;
      q.rows_in = L.nt;
      q.mtiles = 1;
      q.kchunks = L.nt / tc::kTile;
      constexpr int G = 2, S = 3;
      const size_t smem = tc::smem_for<G, S>(q.kchunks);
      e = cudaFuncSetAttribute((const void*)tc::k_tc_contract<G, S>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const int64_t groups = (L.K + G - 1) / G;
      const int grid = (int)std::min<int64_t>(groups, sms);
      tc::k_tc_contract<G, S><<<grid, tc::kThreads, smem, s>>>(q);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pat
