// Batched 2D real FFT stages of the operator (Sec. 3.2, Eq. 16 terms (i) and (iii)).
//
// A P-point complex DFT runs as a Stockham auto-sort FFT (Govindaraju et al.,
// SC'08 formulation) over 1-3 passes of radix 2/4/8/16/32, or for P = 3 * 2^k a
// first pass of radix 24 (3 x 8 in registers) then radix 2-8: each thread holds one
// radix-R butterfly in registers, multiplies by exp(-2 pi i r k / (Ns R))
// (twiddles from a host FP64 table staged in shared memory) and writes the
// R outputs to their sorted positions. The first pass can read its inputs
// straight from global memory and the last pass can write its outputs
// straight to global memory (in both cases a vector's consecutive threads touch
// consecutive elements), so shared memory carries each element once between
// passes. The 2D real transform of a zero-padded n x n slice is split in two
// kernels so every global access is contiguous:
//   row pass    two real rows packed as one complex row (a + i b), FFT over x,
//               untangled into the kx in [0, P/2] half spectra of both rows,
//               written transposed: T[s][kx][y]
//   column pass FFT over y of each kx column (only the n data rows are
//               non-zero), written as X[s][kx][ky] = the contraction's layout.
// The inverse runs the mirror image: column inverse FFT keeping the first n
// rows (crop), then a packed complex-to-real row inverse keeping the first n
// columns. No normalisation here: 1/(px py) is folded into the table.
//
// This header holds the kernels and their per-length launchers (FftLen<R, P>,
// declared in fft_len.h); each fft_*.cu file includes it and instantiates the
// launchers for a set of lengths, so the lengths compile in parallel.
#pragma once
#include "fft_len.h"
#include "pat_internal.h"

namespace pat {
namespace {

constexpr int kThreads = 256;

template <int P>
struct RadixPlan;
template <> struct RadixPlan<16>   { static constexpr int NST = 1, RMAX = 16; static constexpr int R[3] = {16, 1, 1}; };
template <> struct RadixPlan<32>   { static constexpr int NST = 2, RMAX = 8;  static constexpr int R[3] = {8, 4, 1}; };
template <> struct RadixPlan<64>   { static constexpr int NST = 2, RMAX = 8;  static constexpr int R[3] = {8, 8, 1}; };
template <> struct RadixPlan<128>  { static constexpr int NST = 2, RMAX = 16; static constexpr int R[3] = {16, 8, 1}; };
template <> struct RadixPlan<256>  { static constexpr int NST = 2, RMAX = 16; static constexpr int R[3] = {16, 16, 1}; };
template <> struct RadixPlan<512>  { static constexpr int NST = 2, RMAX = 32; static constexpr int R[3] = {32, 16, 1}; };
template <> struct RadixPlan<1024> { static constexpr int NST = 2, RMAX = 32; static constexpr int R[3] = {32, 32, 1}; };
// three times a power of two: a 24-point first pass (every later radix divides 24)
template <> struct RadixPlan<24>   { static constexpr int NST = 1, RMAX = 24; static constexpr int R[3] = {24, 1, 1}; };
template <> struct RadixPlan<48>   { static constexpr int NST = 2, RMAX = 24; static constexpr int R[3] = {24, 2, 1}; };
template <> struct RadixPlan<96>   { static constexpr int NST = 2, RMAX = 24; static constexpr int R[3] = {24, 4, 1}; };
template <> struct RadixPlan<192>  { static constexpr int NST = 2, RMAX = 24; static constexpr int R[3] = {24, 8, 1}; };
template <> struct RadixPlan<384>  { static constexpr int NST = 3, RMAX = 24; static constexpr int R[3] = {24, 8, 2}; };
template <> struct RadixPlan<768>  { static constexpr int NST = 3, RMAX = 24; static constexpr int R[3] = {24, 8, 4}; };

template <int P>
struct Shape {
  static constexpr int TPV = P / RadixPlan<P>::RMAX;  // threads per vector
  static constexpr int VPB = kThreads / TPV;           // vectors per block
  // padded vector stride: the extra element puts consecutive vectors in
  // different banks for the transposed (vector-major) accesses of the row kernels
  static constexpr int VSTR = P + P / 16 + 1;
};

// Radix of pass S and the product of the radices before it.
template <int P, int S>
struct PassOf {
  static constexpr int RAD = RadixPlan<P>::R[S];
  static constexpr int NS = S == 0 ? 1 : (S == 1 ? RadixPlan<P>::R[0] : RadixPlan<P>::R[0] * RadixPlan<P>::R[1]);
};

// Shared-memory twiddles, one block per pass S >= 1 laid out [r - 1][k]
// (r in [1, RAD), k in [0, NS)): the RAD - 1 twiddles W_P^(r k P / (NS RAD))
// a thread needs sit at stride NS, and the threads of a vector (consecutive
// k) read consecutive words, free of bank conflicts.
template <int P>
struct TwPlan {
  static constexpr int len(int S) {
    return S >= RadixPlan<P>::NST || S == 0
               ? 0
               : (RadixPlan<P>::R[S] - 1) * (S == 1 ? RadixPlan<P>::R[0]
                                                    : RadixPlan<P>::R[0] * RadixPlan<P>::R[1]);
  }
  static constexpr int OFF1 = 0, OFF2 = len(1);
  static constexpr int TOTAL = len(1) + len(2);
  static constexpr int N = (TOTAL + 1) & ~1;  // even: the work buffers stay 16-byte aligned
};

// One padding slot per 16 elements keeps the radix-16 scatter of the first
// pass (stride 16) free of shared-memory bank conflicts.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// exp(-2 pi i m / 16) for m in [0, 8) (conjugated for the inverse); m is a
// compile-time constant after unrolling, so the switch folds away.
template <typename R, bool INV>
__device__ __forceinline__ cx<R> mul_w16(cx<R> b, int m) {
  const R c1 = (R)0.92387953251128675613;  // cos(pi/8)
  const R s1 = (R)0.38268343236508977173;  // sin(pi/8)
  const R h = (R)0.70710678118654752440;   // sqrt(2)/2
  cx<R> w;
  switch (m) {
    case 0: return b;
    case 4: return INV ? mk<R>(-b.y, b.x) : mk<R>(b.y, -b.x);  // * (+-i)
    case 1: w = mk<R>(c1, -s1); break;
    case 2: w = mk<R>(h, -h); break;
    case 3: w = mk<R>(s1, -c1); break;
    case 5: w = mk<R>(-s1, -c1); break;
    case 6: w = mk<R>(-h, -h); break;
    default: w = mk<R>(-c1, -s1); break;
  }
  if (INV) w.y = -w.y;
  return cmul(b, w);
}

// exp(-2 pi i m / 32) for m in [0, 16) (conjugated for the inverse): even m
// are the 16th roots above; the odd ones from cos / sin of odd multiples of
// pi / 16.
template <typename R, bool INV>
__device__ __forceinline__ cx<R> mul_w32(cx<R> b, int m) {
  if (!(m & 1)) return mul_w16<R, INV>(b, m >> 1);
  const R c1 = (R)0.98078528040323044913;  // cos(pi/16)
  const R s1 = (R)0.19509032201612826785;  // sin(pi/16)
  const R c3 = (R)0.83146961230254523708;  // cos(3 pi/16)
  const R s3 = (R)0.55557023301960222474;  // sin(3 pi/16)
  cx<R> w;
  switch (m) {
    case 1: w = mk<R>(c1, -s1); break;
    case 3: w = mk<R>(c3, -s3); break;
    case 5: w = mk<R>(s3, -c3); break;
    case 7: w = mk<R>(s1, -c1); break;
    case 9: w = mk<R>(-s1, -c1); break;
    case 11: w = mk<R>(-s3, -c3); break;
    case 13: w = mk<R>(-c3, -s3); break;
    default: w = mk<R>(-c1, -s1); break;  // 15
  }
  if (INV) w.y = -w.y;
  return cmul(b, w);
}

template <int N>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// Complex add / subtract, with PAIRED in FP32 as one f32x2 instruction (each
// lane rounded as the scalar operation is, so the values are identical).
template <bool PAIRED, typename R>
__device__ __forceinline__ cx<R> padd(cx<R> a, cx<R> b) {
  if constexpr (PAIRED && sizeof(R) == 4) {
    cx<R> d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
  } else {
    return cadd(a, b);
  }
}
template <bool PAIRED, typename R>
__device__ __forceinline__ cx<R> psub(cx<R> a, cx<R> b) {
  if constexpr (PAIRED && sizeof(R) == 4) {
    cx<R> d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
  } else {
    return csub(a, b);
  }
}

// Butterfly passes of span LEN, 2 LEN, ..., N (compile-time recursion keeps
// every register index constant). With HOUT only outputs [0, N/2) are needed,
// so the last pass forms only the sums.
template <typename R, int N, int LEN, bool INV, bool HOUT = false, bool PAIRED = false>
__device__ __forceinline__ void dit_passes(cx<R>* a) {
#pragma unroll
  for (int i = 0; i < N; i += LEN) {
#pragma unroll
    for (int k = 0; k < LEN / 2; ++k) {
      cx<R> u = a[i + k];
      cx<R> t = mul_w32<R, INV>(a[i + k + LEN / 2], k * (32 / LEN));
      a[i + k] = padd<PAIRED>(u, t);
      if (!(HOUT && LEN == N)) a[i + k + LEN / 2] = psub<PAIRED>(u, t);
    }
  }
  if constexpr (LEN < N) dit_passes<R, N, 2 * LEN, INV, HOUT, PAIRED>(a);
}

// exp(-2 pi i m / 24) for m in [0, 15) (conjugated for the inverse), from
// cos/sin of multiples of 15 degrees; m is a compile-time constant after
// unrolling.
template <typename R, bool INV>
__device__ __forceinline__ cx<R> w24(int m) {
  const R c15 = (R)0.96592582628906828675;  // cos 15 deg = (sqrt 6 + sqrt 2) / 4
  const R s15 = (R)0.25881904510252076235;  // sin 15 deg = (sqrt 6 - sqrt 2) / 4
  const R c30 = (R)0.86602540378443864676;  // cos 30 deg = sqrt 3 / 2
  const R h = (R)0.70710678118654752440;    // cos 45 deg
  R c, sn;
  switch (m) {
    case 0: c = 1; sn = 0; break;
    case 1: c = c15; sn = s15; break;
    case 2: c = c30; sn = (R)0.5; break;
    case 3: c = h; sn = h; break;
    case 4: c = (R)0.5; sn = c30; break;
    case 5: c = s15; sn = c15; break;
    case 6: c = 0; sn = 1; break;
    case 7: c = -s15; sn = c15; break;
    case 8: c = (R)-0.5; sn = c30; break;
    case 9: c = -h; sn = h; break;
    case 10: c = -c30; sn = (R)0.5; break;
    case 11: c = -c15; sn = s15; break;
    case 12: c = -1; sn = 0; break;
    case 13: c = -c15; sn = -s15; break;
    default: c = -c30; sn = (R)-0.5; break;
  }
  return mk<R>(c, INV ? sn : -sn);
}

template <typename R, int N, bool INV, bool ZIN = false, bool HOUT = false, bool PAIRED = false>
__device__ __forceinline__ void dft_reg(cx<R>* a);

// 24-point DFT as 3 x 8 (Cooley-Tukey): n = 3 n1 + n2, k = k1 + 8 k2;
// X[k1 + 8 k2] = sum_{n2} W3^(n2 k2) W24^(n2 k1) DFT8(x[3 n1 + n2])[k1].
// With ZIN (inputs [12, 24) zero) each DFT8 has its upper half zero.
template <typename R, bool INV, bool ZIN = false>
__device__ __forceinline__ void dft24(cx<R>* a) {
  cx<R> y[3][8];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2)
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) y[n2][n1] = a[3 * n1 + n2];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) dft_reg<R, 8, INV, ZIN>(y[n2]);
  const R r3 = (R)0.86602540378443864676;  // sqrt 3 / 2
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    const cx<R> p = y[0][k1];
    const cx<R> q = cmul(y[1][k1], w24<R, INV>(k1));
    const cx<R> r = cmul(y[2][k1], w24<R, INV>(2 * k1));
    // 3-point DFT of (p, q, r): W3 = exp(-+2 pi i / 3) = -1/2 -+ i sqrt(3)/2
    const cx<R> t1 = cadd(q, r), t2 = csub(q, r);
    const cx<R> m = mk<R>(p.x - (R)0.5 * t1.x, p.y - (R)0.5 * t1.y);
    const cx<R> sv = INV ? mk<R>(-r3 * t2.y, r3 * t2.x) : mk<R>(r3 * t2.y, -r3 * t2.x);
    a[k1] = cadd(p, t1);
    a[k1 + 8] = cadd(m, sv);
    a[k1 + 16] = csub(m, sv);
  }
}

// In-register N-point DFT: N = 2, 4, 8, 16, 32 by radix-2 decimation in time,
// N = 24 as 3 x 8. ZIN: inputs [N/2, N) are zero (zero padding), so after
// the bit reversal every odd slot is zero and the span-2 pass is a copy.
// HOUT: only outputs [0, N/2) are used (crop); ignored for N = 24.
template <typename R, int N, bool INV, bool ZIN, bool HOUT, bool PAIRED>
__device__ __forceinline__ void dft_reg(cx<R>* a) {
  if constexpr (N == 24) {
    dft24<R, INV, ZIN>(a);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int j = bitrev<N>(i);
      if (i < j) {
        cx<R> t = a[i];
        a[i] = a[j];
        a[j] = t;
      }
    }
    if constexpr (ZIN && N > 2) {
#pragma unroll
      for (int i = 0; i < N; i += 2) a[i + 1] = a[i];
      dit_passes<R, N, 4, INV, HOUT, PAIRED>(a);
    } else if constexpr (ZIN) {
      a[1] = a[0];
    } else {
      dit_passes<R, N, 2, INV, HOUT, PAIRED>(a);
    }
  }
}

// Pass S of a Stockham FFT of P points on the vector `buf` (shared memory,
// padded indexing). With FROM_LOAD the first pass reads element i as ld(i)
// instead of from buf; with TO_STORE the last pass hands element i to st(i, v)
// instead of writing buf (in the last pass the output index is j + r Ns, so a
// vector's consecutive threads store consecutive elements). Every thread of the
// block calls every pass (they hold __syncthreads).
//
// ZIN: elements [P/2, P) of the input are zero (the zero padding of a slice of
// at most P/2 rows or columns): the first pass, whose element r is
// j + r P/RAD, neither reads nor adds its upper RAD/2 elements. HOUT: only
// outputs [0, P/2) are used (the crop): the last pass, whose element r is
// j + r P/RAD, neither forms nor writes its upper RAD/2 outputs (with a
// shared-memory last pass those slots keep stale values).
template <typename R, int P, int S, bool INV, bool FROM_LOAD, bool TO_STORE, bool ZIN = false,
          bool HOUT = false, class LD, class ST>
__device__ __forceinline__ void run_passes(cx<R>* buf, const cx<R>* tw, int tid, LD& ld, ST& st) {
  constexpr int NST = RadixPlan<P>::NST;
  constexpr int RAD = PassOf<P, S>::RAD;
  constexpr int NS = PassOf<P, S>::NS;
  constexpr int TPV = Shape<P>::TPV;
  constexpr int NB = P / RAD;
  constexpr int PER = NB / TPV;
  constexpr bool first_ld = FROM_LOAD && S == 0;
  constexpr bool last_st = TO_STORE && S == NST - 1;
  constexpr bool zin = ZIN && S == 0;
  constexpr bool hout = HOUT && S == NST - 1;
  constexpr int RIN = zin ? RAD / 2 : RAD;    // elements read
  constexpr int ROUT = hout ? RAD / 2 : RAD;  // outputs kept
  cx<R> v[PER][RAD];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * TPV;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      if (r >= RIN)
        v[q][r] = mk<R>(0, 0);
      else if constexpr (first_ld)
        v[q][r] = ld(j + r * NB);
      else
        v[q][r] = buf[pidx(j + r * NB)];
    }
    if constexpr (NS > 1) {
      const int k = j % NS;
      const cx<R>* tws = tw + (S == 1 ? TwPlan<P>::OFF1 : TwPlan<P>::OFF2) + k;
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        cx<R> w = tws[(r - 1) * NS];
        if (INV) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
    }
    // paired FP32 adds in the radix-2 butterflies of the plans with radices up
    // to 16 (P <= 256: measured faster; the radix-32 and 3 * 2^k plans were
    // slower with them and keep scalar adds)
    dft_reg<R, RAD, INV, zin, hout, (RadixPlan<P>::RMAX <= 16)>(v[q]);
  }
  if constexpr (last_st) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = tid + q * TPV;  // j < NS in the last pass: base index = j
#pragma unroll
      for (int r = 0; r < ROUT; ++r) st(j + r * NS, v[q][r]);
    }
  } else {
    if constexpr (!first_ld) __syncthreads();  // in place: every read before any write
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = tid + q * TPV;
      const int k = j % NS;
      const int base = (j - k) * RAD + k;
#pragma unroll
      for (int r = 0; r < ROUT; ++r) buf[pidx(base + r * NS)] = v[q][r];
    }
    __syncthreads();
  }
  if constexpr (S + 1 < NST)
    run_passes<R, P, S + 1, INV, FROM_LOAD, TO_STORE, ZIN, HOUT>(buf, tw, tid, ld, st);
}

template <typename R>
struct SmemLoad {  // unused placeholder type for passes that read buf
  __device__ cx<R> operator()(int) const { return mk<R>(0, 0); }
};
template <typename R>
struct NoStore {
  __device__ void operator()(int, cx<R>) const {}
};

template <typename R, int P>
__device__ __forceinline__ cx<R>* setup_smem(const cx<R>* tw_g, cx<R>** tw_s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using TP = TwPlan<P>;
  cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
  for (int i = threadIdx.x; i < TP::TOTAL; i += blockDim.x) {
    const bool second = i >= TP::OFF2;
    const int rem = second ? i - TP::OFF2 : i;
    constexpr int NS1 = PassOf<P, 1>::NS, RAD1 = PassOf<P, 1>::RAD;
    constexpr int NS2 = RadixPlan<P>::NST > 2 ? PassOf<P, 2>::NS : 1;
    constexpr int RAD2 = RadixPlan<P>::NST > 2 ? PassOf<P, 2>::RAD : 1;
    const int ns = second ? NS2 : NS1;
    const int r = rem / ns + 1, k = rem % ns;
    const int step = second ? P / (NS2 * RAD2) : P / (NS1 * RAD1);
    tw[i] = tw_g[r * k * step];  // r k < NS RAD: index < P
  }
  *tw_s = tw;
  return tw + TP::N;
}

template <typename R, int P>
constexpr size_t smem_bytes() {
  return sizeof(cx<R>) * (size_t)(TwPlan<P>::N + Shape<P>::VPB * Shape<P>::VSTR);
}

// Compact index of sensor coordinate c on a scan axis (offset o, stride st,
// n samples), or -1 when c is not a scan position.
__device__ __forceinline__ int scan_index(int c, int o, int st, int n) {
  const int d = c - o;
  if (d < 0 || d % st) return -1;
  const int i = d / st;
  return i < n ? i : -1;
}

// Input of one packed row pair (rows y0, y0 + 1 of a slice, a + i b),
// zero-padded from nx_in: the plain [ny][nx] slice, or with SAMP the
// zero-filled image of scan-grid data [my][mx] (the adjoint of the measurement
// operator, Sec. 3.3). Rows at or past ny_in read as zero.
template <typename R, bool SAMP>
struct RowPairLoad {
  const R* row0;
  const R* row1;
  bool ok0, ok1;
  int nx_in;
  Samp sm;
  __device__ __forceinline__ RowPairLoad(const R* base, int y0, int nx, int ny_in, Samp s)
      : nx_in(nx), sm(s) {
    if (!SAMP) {
      ok0 = y0 < ny_in;
      ok1 = y0 + 1 < ny_in;
      row0 = base + (int64_t)y0 * nx_in;
      row1 = row0 + nx_in;
    } else {
      const int j0 = y0 < ny_in ? scan_index(y0, sm.oy, sm.sy, sm.my) : -1;
      const int j1 = y0 + 1 < ny_in ? scan_index(y0 + 1, sm.oy, sm.sy, sm.my) : -1;
      ok0 = j0 >= 0;
      ok1 = j1 >= 0;
      row0 = base + (int64_t)(ok0 ? j0 : 0) * sm.mx;
      row1 = base + (int64_t)(ok1 ? j1 : 0) * sm.mx;
    }
  }
  __device__ __forceinline__ cx<R> operator()(int x) const {
    R a = 0, b = 0;
    if (x < nx_in) {
      int xi = x;
      if (SAMP) xi = scan_index(x, sm.ox, sm.sx, sm.mx);
      if (xi >= 0) {
        if (ok0) a = row0[xi];
        if (ok1) b = row1[xi];
      }
    }
    return mk<R>(a, b);
  }
};

// Output of one row pair of an image slice from the packed inverse transform
// (Re -> row y0, Im -> row y0 + 1), columns [0, nx_out) kept; with `sub`,
// writes image - sub and accumulates its squares (FP64) in acc. With SAMP
// only the scan positions are kept, written compactly to [my][mx] (the
// measurement operator of Sec. 3.3); `sub` has that layout. Rows at or past
// ny_out are not written.
template <typename R, bool SAMP>
struct RowPairStore {
  R* dslice;
  const R* sslice;
  int64_t off0, off1;
  bool ok0, ok1;
  int nx_out;
  Samp sm;
  double acc = 0.0;
  __device__ __forceinline__ RowPairStore(R* out_slice, const R* sub_slice, int y0, int nx,
                                          int ny_out, Samp s)
      : dslice(out_slice), sslice(sub_slice), nx_out(nx), sm(s) {
    if (!SAMP) {
      ok0 = y0 < ny_out;
      ok1 = y0 + 1 < ny_out;
      off0 = (int64_t)y0 * nx_out;
      off1 = off0 + nx_out;
    } else {
      const int j0 = y0 < ny_out ? scan_index(y0, sm.oy, sm.sy, sm.my) : -1;
      const int j1 = y0 + 1 < ny_out ? scan_index(y0 + 1, sm.oy, sm.sy, sm.my) : -1;
      ok0 = j0 >= 0;
      ok1 = j1 >= 0;
      off0 = (int64_t)(ok0 ? j0 : 0) * sm.mx;
      off1 = (int64_t)(ok1 ? j1 : 0) * sm.mx;
    }
  }
  __device__ __forceinline__ void operator()(int x, cx<R> z) {
    if (x >= nx_out) return;
    int xi = x;
    if (SAMP) {
      xi = scan_index(x, sm.ox, sm.sx, sm.mx);
      if (xi < 0) return;
    }
    if (ok0) {
      R r0 = z.x;
      if (sslice) {
        r0 -= sslice[off0 + xi];
        acc += (double)r0 * (double)r0;
      }
      dslice[off0 + xi] = r0;
    }
    if (ok1) {
      R r1 = z.y;
      if (sslice) {
        r1 -= sslice[off1 + xi];
        acc += (double)r1 * (double)r1;
      }
      dslice[off1 + xi] = r1;
    }
  }
};

// Deterministic block sum of acc (warp shuffle tree, then warp 0 over the
// warps) written by thread 0 to *dst. Every thread of the block calls it.
__device__ __forceinline__ void block_sum_to(double acc, double* dst) {
  __shared__ double wsum[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < kThreads / 32 ? wsum[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) *dst = w;
  }
}

// Row pair (A, B) of half spectra at kx from the transform Z of the packed
// pair a + i b: A = (Z + conj Zm) / 2, B = (Z - conj Zm) / (2i), Zm = Z[P - kx].
template <typename R>
__device__ __forceinline__ void untangle(cx<R> Z, cx<R> Zm, cx<R>* A, cx<R>* B) {
  *A = mk<R>((R)0.5 * (Z.x + Zm.x), (R)0.5 * (Z.y - Zm.y));
  *B = mk<R>((R)0.5 * (Z.y + Zm.y), (R)-0.5 * (Z.x - Zm.x));
}

// Adjacent pair T[kx][y], T[kx][y + 1] (y even, row stride even, so the
// pair is 16-byte aligned in FP32) as one vector access.
template <typename R>
__device__ __forceinline__ void load_pair(const cx<R>* p, cx<R>* a, cx<R>* b) {
  if constexpr (sizeof(R) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    *a = mk<R>(v.x, v.y);
    *b = mk<R>(v.z, v.w);
  } else {
    *a = p[0];
    *b = p[1];
  }
}
template <typename R>
__device__ __forceinline__ void store_pair(cx<R>* p, cx<R> a, cx<R> b) {
  if constexpr (sizeof(R) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// Inverse of untangle, written into a packed vector: Z[kx] = A + i B and
// Z[P - kx] = conj(A) + i conj(B) (A, B the half spectra of two real rows).
template <typename R, int P>
__device__ __forceinline__ void pack_pair(cx<R>* b, int kx, cx<R> A, cx<R> B) {
  b[pidx(kx)] = mk<R>(A.x - B.y, A.y + B.x);
  if (kx > 0 && kx < P / 2) b[pidx(P - kx)] = mk<R>(A.x + B.y, B.x - A.y);
}

// Stage i, row pass: rows y0 = 2 pair, y0 + 1 of slice s packed as a + i b,
// zero-padded from nx_in to P, transformed; half spectra written to
// T[s][kx][y] for kx in [0, P/2]. With sampling on, the slice is the
// zero-filled image of scan-grid data in[s][my][mx] (the adjoint of the
// measurement operator, Sec. 3.3).
template <typename R, int P, bool SAMP, bool ZIN>
__global__ void __launch_bounds__(kThreads) k_row_r2c(const R* __restrict__ in, int64_t in_stride,
                                                      int nx_in, int ny_in, cx<R>* __restrict__ T,
                                                      int tstride, int64_t tslice,
                                                      const cx<R>* __restrict__ tw_g, Samp sm) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t s = blockIdx.y;
  const int pair0 = blockIdx.x * SH::VPB;
  RowPairLoad<R, SAMP> ld(in + s * in_stride, 2 * (pair0 + v), nx_in, ny_in, sm);
  pdl_wait();
  __syncthreads();  // twiddles staged
  NoStore<R> st;
  run_passes<R, P, 0, false, true, false, ZIN>(bufs + v * SH::VSTR, tw, tid, ld, st);
  cx<R>* dst = T + s * tslice;
#pragma unroll 4
  for (int i = threadIdx.x; i < SH::VPB * (P / 2 + 1); i += kThreads) {
    const int vv = i % SH::VPB, kx = i / SH::VPB;
    const int yy = 2 * (pair0 + vv);
    if (yy >= ny_in) continue;
    cx<R> A, B;
    untangle(bufs[vv * SH::VSTR + pidx(kx)], bufs[vv * SH::VSTR + pidx((P - kx) % P)], &A,
             &B);
    store_pair(dst + (int64_t)kx * tstride + yy, A, B);  // tstride even: yy + 1 < tstride
  }
}

// The bins ky and P - ky of one column (mirror pair) sit in adjacent slots
// of the representative-slot layout (members 0 / 1 or 2 / 3 of one D4
// representative), so a slot-mapped column stores them as one 16-byte access
// when their slots are an aligned pair, else as two.
template <typename R>
__device__ __forceinline__ void slot_store_pair(cx<R>* dst, int s0, int s1, cx<R> v0, cx<R> v1) {
  if (s1 == s0 + 1 && !(s0 & 1)) {
    store_pair(dst + s0, v0, v1);
  } else if (s0 == s1 + 1 && !(s1 & 1)) {
    store_pair(dst + s1, v1, v0);
  } else {
    dst[s0] = v0;
    dst[s1] = v1;
  }
}

// Stage i, column pass: T[s][kx][0..n_in) zero-padded to P, FFT over y,
// written to out[s][kx][0..P) (slice stride out_stride), or with `slot` to
// out[s][slot[kx * P + ky]] (the representative-slot layout; the transform
// then lands in the work vector and leaves as mirror pairs).
template <typename R, int P, bool SLOT, bool ZIN>
__global__ void __launch_bounds__(kThreads) k_col_fwd(const cx<R>* __restrict__ T, int tstride,
                                                      int64_t tslice, int n_in, int ncols,
                                                      int64_t nvec, cx<R>* __restrict__ out,
                                                      int64_t out_stride,
                                                      const cx<R>* __restrict__ tw_g,
                                                      const int* __restrict__ slot) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t g = (int64_t)blockIdx.x * SH::VPB + v;
  const bool ok = g < nvec;
  // 32-bit quotient (nvec = slices x columns < 2^31): no 64-bit division
  const unsigned gq = ok ? (unsigned)g / (unsigned)ncols : 0u;
  const int64_t s = gq, kx = ok ? (int64_t)((unsigned)g - gq * (unsigned)ncols) : 0;
  const cx<R>* src = T + s * tslice + kx * tstride;
  cx<R>* dst = out + s * out_stride;
  const int* sl = SLOT ? slot + kx * P : nullptr;
  pdl_wait();
  __syncthreads();
  auto ld = [&](int y) -> cx<R> { return (ok && y < n_in) ? src[y] : mk<R>(0, 0); };
  if constexpr (SLOT) {
    cx<R>* b = bufs + v * SH::VSTR;
    NoStore<R> ns;
    run_passes<R, P, 0, false, true, false, ZIN>(b, tw, tid, ld, ns);  // ends with a barrier
    if (ok) {
#pragma unroll
      for (int i = 0; i < (P / 2 + SH::TPV) / SH::TPV; ++i) {
        const int y = tid + i * SH::TPV;
        if (y > P / 2) break;
        const int s0 = __ldg(sl + y);
        if (y == 0 || y == P / 2) {
          dst[s0] = b[pidx(y)];
          continue;
        }
        slot_store_pair(dst, s0, __ldg(sl + P - y), b[pidx(y)], b[pidx(P - y)]);
      }
    }
  } else {
    auto st = [&](int y, cx<R> val) {
      if (ok) dst[kx * P + y] = val;
    };
    run_passes<R, P, 0, false, true, true, ZIN>(bufs + v * SH::VSTR, tw, tid, ld, st);
  }
}

// Stage iii, column pass: in[s][kx][0..P) (or with `slot`, in[s][slot[kx * P +
// ky]]) inverse FFT over ky, rows [0, n_out) kept (crop) into T[s][kx][y].
template <typename R, int P, bool SLOT, bool HOUT>
__global__ void __launch_bounds__(kThreads) k_col_inv(const cx<R>* __restrict__ in,
                                                      int64_t in_stride, int ncols, int64_t nvec,
                                                      cx<R>* __restrict__ T, int tstride,
                                                      int64_t tslice, int n_out,
                                                      const cx<R>* __restrict__ tw_g,
                                                      const int* __restrict__ slot) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t g = (int64_t)blockIdx.x * SH::VPB + v;
  const bool ok = g < nvec;
  // 32-bit quotient (nvec = slices x columns < 2^31): no 64-bit division
  const unsigned gq = ok ? (unsigned)g / (unsigned)ncols : 0u;
  const int64_t s = gq, kx = ok ? (int64_t)((unsigned)g - gq * (unsigned)ncols) : 0;
  const cx<R>* src = in + s * in_stride;
  const int* sl = SLOT ? slot + kx * P : nullptr;
  cx<R>* dst = T + s * tslice + kx * tstride;
  pdl_wait();
  __syncthreads();
  auto ld = [&](int y) -> cx<R> {
    return ok ? src[SLOT ? __ldg(sl + y) : kx * P + y] : mk<R>(0, 0);
  };
  auto st = [&](int y, cx<R> val) {
    if (ok && y < n_out) dst[y] = val;
  };
  // (slot-mapped columns load element by element here: gathering mirror
  // pairs as 16-byte loads through the work vector measured slower)
  run_passes<R, P, 0, true, true, true, false, HOUT>(bufs + v * SH::VSTR, tw, tid, ld, st);
}

// Stage iii row pass, first half: the half spectra A = T[kx][y0], B =
// T[kx][y0 + 1] of the block's VPB row pairs, packed Hermitian-extended into
// the work vectors. All global loads first (independent, in flight
// together), then the packing into shared memory.
template <typename R, int P>
__device__ __forceinline__ void load_packed_pairs(const cx<R>* __restrict__ src, int tstride,
                                                  int pair0, int ny_out, cx<R>* bufs) {
  using SH = Shape<P>;
  constexpr int NH = SH::VPB * (P / 2 + 1);
  constexpr int NIT = (NH + kThreads - 1) / kThreads;
  // loads in flight per thread: all of them in FP32 (one 16-byte load per pair)
  constexpr int CH = sizeof(R) == 4 ? (NIT <= 13 ? NIT : 8) : 4;
#pragma unroll
  for (int c0 = 0; c0 < NIT; c0 += CH) {
    cx<R> Av[CH], Bv[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int i = threadIdx.x + (c0 + c) * kThreads;
      const int vv = i % SH::VPB, kx = i / SH::VPB;
      const int yy = 2 * (pair0 + vv);
      Av[c] = mk<R>(0, 0);
      Bv[c] = mk<R>(0, 0);
      if (c0 + c < NIT && i < NH && yy < ny_out) {
        // the pair's second element exists even for odd ny_out (row stride even)
        load_pair(src + (int64_t)kx * tstride + yy, &Av[c], &Bv[c]);
        if (yy + 1 >= ny_out) Bv[c] = mk<R>(0, 0);
      }
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int i = threadIdx.x + (c0 + c) * kThreads;
      if (c0 + c >= NIT || i >= NH) break;
      const int vv = i % SH::VPB, kx = i / SH::VPB;
      cx<R> A = Av[c], B = Bv[c];
      if (kx == 0 || kx == P / 2) {  // spectra of real rows: real at DC and Nyquist
        A.y = 0;
        B.y = 0;
      }
      pack_pair<R, P>(bufs + vv * SH::VSTR, kx, A, B);
    }
  }
}

// Stage iii, row pass: half spectra A = T[s][kx][y0], B = T[s][kx][y0 + 1]
// of two real rows, packed as Z = A + iB with the Hermitian extension
// Z[P - kx] = conj(A) + i conj(B), inverse FFT over x; Re -> row y0,
// Im -> row y0 + 1, columns [0, nx_out) kept. With `sub`, writes
// image - sub and accumulates its squares (FP64) per block into partials.
// With sampling on, only the scan positions are kept, written compactly to
// out[s][my][mx] (the measurement operator of Sec. 3.3); `sub` has that layout.
template <typename R, int P, bool SAMP, bool HOUT>
__global__ void __launch_bounds__(kThreads) k_row_c2r(const cx<R>* __restrict__ T, int tstride,
                                                      int64_t tslice, int nx_out, int ny_out,
                                                      R* __restrict__ out, int64_t out_stride,
                                                      const R* __restrict__ sub,
                                                      double* __restrict__ partials,
                                                      const cx<R>* __restrict__ tw_g, Samp sm) {
  using SH = Shape<P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t s = blockIdx.y;
  const int pair0 = blockIdx.x * SH::VPB;
  const cx<R>* src = T + s * tslice;
  pdl_wait();
  load_packed_pairs<R, P>(src, tstride, pair0, ny_out, bufs);
  __syncthreads();
  RowPairStore<R, SAMP> st(out + s * out_stride, sub ? sub + s * out_stride : nullptr,
                           2 * (pair0 + v), nx_out, ny_out, sm);
  SmemLoad<R> ld;
  run_passes<R, P, 0, true, false, true, false, HOUT>(bufs + v * SH::VSTR, tw, tid, ld, st);
  if (partials) block_sum_to(st.acc, partials + (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// The residual pass stages the measured rows of its block in shared memory
// (single precision, unsampled data: 2 VPB rows of at most P/2 floats after
// the work vectors), where that keeps 4 CTAs per SM (<= 56 KB). The data of a
// solve are written before its first kernel runs, so the copies are issued
// before the dependency wait and overlap the previous kernel's end and this
// kernel's spectrum loads.
template <typename R, int P, bool SAMP>
struct ResidStage {
  static constexpr size_t rows_bytes = sizeof(R) * 2 * Shape<P>::VPB * (P / 2);
  static constexpr bool on =
      !SAMP && sizeof(R) == 4 && smem_bytes<R, P>() + rows_bytes <= 56 * 1024;
  static constexpr size_t bytes = on ? rows_bytes : 0;
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// The step pass stages the FISTA state (y_k and x_{k-1}) of its rows the
// same way, where that keeps 3 CTAs per SM (<= 76 KB): written by the
// previous iteration's step pass (or before the first kernel of the solve),
// it is visible before the dependency wait.
template <typename R, int P>
struct StepStage {
  static constexpr size_t rows_bytes = sizeof(R) * 2 * Shape<P>::VPB * (P / 2);
  static constexpr bool on = sizeof(R) == 4 && smem_bytes<R, P>() + 2 * rows_bytes <= 76 * 1024;
  static constexpr size_t bytes = on ? 2 * rows_bytes : 0;
};

// Copies n floats from global src to shared dst (16-byte copies when both the
// source and the count allow, else 4-byte copies); the block's threads share
// the work. Waited for by cp_async_wait_all.
template <typename R>
__device__ __forceinline__ void stage_rows(R* dst, const R* src, int n) {
  if (((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (n & 3) == 0) {
    for (int i = 4 * threadIdx.x; i < n; i += 4 * kThreads) cp_async16(dst + i, src + i);
  } else {
    for (int i = threadIdx.x; i < n; i += kThreads) cp_async4(dst + i, src + i);
  }
}

// Residual row pass between H and H* (the gradient of Eq. 15): for the
// block's row pairs of slice s, the inverse row transform as k_row_c2r does
// it, then r = image - y at the kept (scan) positions and zero elsewhere, its
// squares summed in FP64 into partials, then the forward row transform of r as
// k_row_r2c does it, its half spectra written back over the same rows of T
// (each block reads its rows entirely before writing them). The residual
// itself never leaves the chip. With `total`, the last block to finish (block
// counter `count`, zero on entry and re-armed) also sums the partials into
// *total. A plan's nx is at most P/2 (P >= 2 nx - 1,
// P even), so the inverse transform forms only x < P/2 and the forward one
// skips the zero half.
template <typename R, int P, bool SAMP>
__global__ void __launch_bounds__(kThreads) k_row_resid(cx<R>* __restrict__ T, int tstride,
                                                        int64_t tslice, int nx, int ny,
                                                        const R* __restrict__ y,
                                                        int64_t y_stride,
                                                        double* __restrict__ partials,
                                                        double* __restrict__ total,
                                                        unsigned* __restrict__ count,
                                                        const cx<R>* __restrict__ tw_g, Samp sm) {
  using SH = Shape<P>;
  using YS = ResidStage<R, P, SAMP>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t s = blockIdx.y;
  const int pair0 = blockIdx.x * SH::VPB;
  cx<R>* Ts = T + s * tslice;
  // rows [2 pair0, 2 pair0 + nrows) of the measured slice, contiguous
  R* ys = reinterpret_cast<R*>(bufs + SH::VPB * SH::VSTR);
  if constexpr (YS::on)
    stage_rows(ys, y + s * y_stride + (int64_t)(2 * pair0) * nx,
               min(2 * SH::VPB, ny - 2 * pair0) * nx);
  pdl_wait();
  load_packed_pairs<R, P>(Ts, tstride, pair0, ny, bufs);
  if constexpr (YS::on) cp_async_wait_all();
  __syncthreads();
  cx<R>* b = bufs + v * SH::VSTR;
  SmemLoad<R> sl;
  NoStore<R> ns;
  // the layout of y: the row pair's offsets (scan rows with sampling on)
  const int y0 = 2 * (pair0 + v);
  RowPairStore<R, SAMP> rows(nullptr, y + s * y_stride, y0, nx, ny, sm);
  double acc = 0.0;
  // image rows x < P/2 from the last inverse pass, turned into the residual
  // in place: that pass writes exactly the positions its thread read, so r
  // replaces the image without a barrier (zero past nx; the forward pass
  // below does not read x >= P/2)
  auto resid = [&](int x, cx<R> z) {
    R r0 = 0, r1 = 0;
    int xi = x < nx ? x : -1;
    if (SAMP && xi >= 0) xi = scan_index(x, sm.ox, sm.sx, sm.mx);
    if (xi >= 0) {
      if (rows.ok0) {
        r0 = z.x - (YS::on ? ys[2 * v * nx + xi] : rows.sslice[rows.off0 + xi]);
        acc += (double)r0 * (double)r0;
      }
      if (rows.ok1) {
        r1 = z.y - (YS::on ? ys[(2 * v + 1) * nx + xi] : rows.sslice[rows.off1 + xi]);
        acc += (double)r1 * (double)r1;
      }
    }
    b[pidx(x)] = mk<R>(r0, r1);
  };
  run_passes<R, P, 0, true, false, true, false, true>(b, tw, tid, sl, resid);
  __syncthreads();
  run_passes<R, P, 0, false, false, false, true>(b, tw, tid, sl, ns);  // spectrum of r0 + i r1
#pragma unroll 4
  for (int i = threadIdx.x; i < SH::VPB * (P / 2 + 1); i += kThreads) {
    const int vv = i % SH::VPB, kx = i / SH::VPB;
    const int yy = 2 * (pair0 + vv);
    if (yy >= ny) continue;
    cx<R> A, B;
    untangle(bufs[vv * SH::VSTR + pidx(kx)], bufs[vv * SH::VSTR + pidx((P - kx) % P)], &A,
             &B);
    store_pair(Ts + (int64_t)kx * tstride + yy, A, B);  // tstride even: yy + 1 < tstride
  }
  if (partials) block_sum_to(acc, partials + (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
  if (total) {
    // the last block to finish sums every block's partial in a fixed order
    // into *total (FP64, deterministic) and re-arms the counter
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(count, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const int n = (int)(gridDim.x * gridDim.y);
      double sum = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) sum += __ldcg(partials + i);
      block_sum_to(sum, total);
      if (threadIdx.x == 0) *count = 0u;
    }
  }
}

// Stage iii row pass over the depth slices with the FISTA step (Eq. 14-15)
// in place of the gradient store: each gradient value g of the kept columns
// updates y (momentum point) and xprev (x_{k-1}) of its voxel in place; the
// last block to finish advances the iteration (see FistaStep). Only x < P/2
// is formed (a plan's nx is at most P/2). With NEXT the block then takes the
// new momentum point y_{k+1} of its rows through the forward row transform
// of stage i (as k_row_r2c does) and writes it over the same rows of T, so
// the next iteration's stage i is its column pass alone.
template <typename R, int P, bool NEXT>
__global__ void __launch_bounds__(kThreads) k_row_c2r_step(
    cx<R>* __restrict__ T, int tstride, int64_t tslice, int nx, int ny, int64_t plane,
    R* __restrict__ yv, R* __restrict__ xprev, const double* __restrict__ scal,
    const double* __restrict__ betas, int* __restrict__ iter, const double* __restrict__ r2_cur,
    double* __restrict__ r2_hist, int cap, unsigned* __restrict__ done,
    const cx<R>* __restrict__ tw_g) {
  using SH = Shape<P>;
  using SS = StepStage<R, P>;
  cx<R>* tw;
  cx<R>* bufs = setup_smem<R, P>(tw_g, &tw);
  const int v = threadIdx.x / SH::TPV, tid = threadIdx.x % SH::TPV;
  const int64_t s = blockIdx.y;
  const int pair0 = blockIdx.x * SH::VPB;
  // y_k and x_{k-1} of rows [2 pair0, 2 pair0 + 2 VPB), staged after the work vectors
  R* sy = reinterpret_cast<R*>(bufs + SH::VPB * SH::VSTR);
  R* sx = sy + 2 * SH::VPB * (P / 2);
  if constexpr (SS::on) {
    const int n = min(2 * SH::VPB, ny - 2 * pair0) * nx;
    stage_rows(sy, yv + s * plane + (int64_t)(2 * pair0) * nx, n);
    stage_rows(sx, xprev + s * plane + (int64_t)(2 * pair0) * nx, n);
  }
  pdl_wait();
  const R invL = (R)scal[0], lamL = (R)scal[1];
  const int k = *iter;
  const R beta = (R)betas[k];
  load_packed_pairs<R, P>(T + s * tslice, tstride, pair0, ny, bufs);
  if constexpr (SS::on) cp_async_wait_all();
  __syncthreads();
  const int y0 = 2 * (pair0 + v);
  const bool ok0 = y0 < ny, ok1 = y0 + 1 < ny;
  R* ys = yv + s * plane + (int64_t)y0 * nx;
  R* xs = xprev + s * plane + (int64_t)y0 * nx;
  const R* syv = sy + 2 * v * nx;  // this pair's staged rows (i in [0, 2 nx))
  const R* sxv = sx + 2 * v * nx;
  auto upd = [&](int64_t i, R g) -> R {
    const R ya = SS::on ? syv[i] : ys[i], xp = SS::on ? sxv[i] : xs[i];
    R x = ya - g * invL - lamL;
    x = x > (R)0 ? x : (R)0;
    const R yn = x + beta * (x - xp);
    ys[i] = yn;
    xs[i] = x;
    return yn;
  };
  cx<R>* b = bufs + v * SH::VSTR;
  // the last inverse pass writes exactly the positions its thread read, so
  // with NEXT the new momentum point y_{k+1} (rows y0 + i y0 + 1, zero past
  // nx) replaces the gradient in place as the next forward transform's input
  auto st = [&](int x, cx<R> z) {
    R n0 = 0, n1 = 0;
    if (x < nx) {
      if (ok0) n0 = upd(x, z.x);
      if (ok1) n1 = upd((int64_t)nx + x, z.y);
    }
    if constexpr (NEXT) b[pidx(x)] = mk<R>(n0, n1);
  };
  SmemLoad<R> ld;
  run_passes<R, P, 0, true, false, true, false, true>(b, tw, tid, ld, st);
  if constexpr (NEXT) {
    __syncthreads();
    NoStore<R> ns;
    run_passes<R, P, 0, false, false, false, true>(b, tw, tid, ld, ns);  // zero half skipped
    cx<R>* Ts = T + s * tslice;
#pragma unroll 4
    for (int i = threadIdx.x; i < SH::VPB * (P / 2 + 1); i += kThreads) {
      const int vv = i % SH::VPB, kx = i / SH::VPB;
      const int yy = 2 * (pair0 + vv);
      if (yy >= ny) continue;
      cx<R> A, B;
      untangle(bufs[vv * SH::VSTR + pidx(kx)], bufs[vv * SH::VSTR + pidx((P - kx) % P)], &A, &B);
      store_pair(Ts + (int64_t)kx * tstride + yy, A, B);  // tstride even: yy + 1 < tstride
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    if (k < cap) r2_hist[k] = *r2_cur;
    *iter = k + 1;
    *done = 0;
  }
}

template <typename R, int P>
cudaError_t set_smem_attr(const void* fn) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<R, P>());
}
}  // namespace

// ---- launchers, one per stage and length ---------------------------------------
template <typename R, int P>
cudaError_t FftLen<R, P>::row_r2c(const R* in, int64_t in_stride, int nx_in, int ny_in, cx<R>* T, int tstride,
                                  int64_t tslice, int S, const cx<R>* tw, cudaStream_t st, Samp sm) {
  using SH = Shape<P>;
  const bool zin = 2 * nx_in <= P;  // the zero padding covers [P/2, P)
  auto fn = sm.on ? (zin ? k_row_r2c<R, P, true, true> : k_row_r2c<R, P, true, false>)
                  : (zin ? k_row_r2c<R, P, false, true> : k_row_r2c<R, P, false, false>);
  cudaError_t e = set_smem_attr<R, P>((const void*)fn);
  if (e != cudaSuccess) return e;
  const int pairs = (ny_in + 1) / 2;
  dim3 grid((pairs + SH::VPB - 1) / SH::VPB, S);
  return launch_pdl(fn, grid, dim3(kThreads), smem_bytes<R, P>(), st, in, in_stride, nx_in, ny_in,
                    T, tstride, tslice, tw, sm);
}

template <typename R, int P>
cudaError_t FftLen<R, P>::col_fwd(const cx<R>* T, int tstride, int64_t tslice, int n_in, int ncols, int S,
                                  cx<R>* out, int64_t out_stride, const cx<R>* tw, cudaStream_t st,
                                  const int* slot) {
  using SH = Shape<P>;
  const bool zin = 2 * n_in <= P;
  auto fn = slot ? (zin ? k_col_fwd<R, P, true, true> : k_col_fwd<R, P, true, false>)
                 : (zin ? k_col_fwd<R, P, false, true> : k_col_fwd<R, P, false, false>);
  cudaError_t e = set_smem_attr<R, P>((const void*)fn);
  if (e != cudaSuccess) return e;
  const int64_t nvec = (int64_t)S * ncols;
  const int64_t blocks = (nvec + SH::VPB - 1) / SH::VPB;
  return launch_pdl(fn, dim3((unsigned)blocks), dim3(kThreads), smem_bytes<R, P>(), st,
                    T, tstride, tslice, n_in, ncols, nvec, out, out_stride, tw, slot);
}

template <typename R, int P>
cudaError_t FftLen<R, P>::col_inv(const cx<R>* in, int64_t in_stride, int ncols, int S, cx<R>* T, int tstride,
                                  int64_t tslice, int n_out, const cx<R>* tw, cudaStream_t st, const int* slot) {
  using SH = Shape<P>;
  const bool hout = 2 * n_out <= P;  // rows [P/2, P) are cropped away
  auto fn = slot ? (hout ? k_col_inv<R, P, true, true> : k_col_inv<R, P, true, false>)
                 : (hout ? k_col_inv<R, P, false, true> : k_col_inv<R, P, false, false>);
  cudaError_t e = set_smem_attr<R, P>((const void*)fn);
  if (e != cudaSuccess) return e;
  const int64_t nvec = (int64_t)S * ncols;
  const int64_t blocks = (nvec + SH::VPB - 1) / SH::VPB;
  return launch_pdl(fn, dim3((unsigned)blocks), dim3(kThreads), smem_bytes<R, P>(), st,
                    in, in_stride, ncols, nvec, T, tstride, tslice, n_out, tw, slot);
}

template <typename R, int P>
cudaError_t FftLen<R, P>::row_c2r(const cx<R>* T, int tstride, int64_t tslice, int nx_out, int ny_out, R* out,
                                  int64_t out_stride, int S, const R* sub, double* partials, const cx<R>* tw,
                                  cudaStream_t st, int* nblocks, Samp sm) {
  using SH = Shape<P>;
  const bool hout = 2 * nx_out <= P;
  auto fn = sm.on ? (hout ? k_row_c2r<R, P, true, true> : k_row_c2r<R, P, true, false>)
                  : (hout ? k_row_c2r<R, P, false, true> : k_row_c2r<R, P, false, false>);
  cudaError_t e = set_smem_attr<R, P>((const void*)fn);
  if (e != cudaSuccess) return e;
  const int pairs = (ny_out + 1) / 2;
  dim3 grid((pairs + SH::VPB - 1) / SH::VPB, S);
  *nblocks = (int)(grid.x * grid.y);
  return launch_pdl(fn, grid, dim3(kThreads), smem_bytes<R, P>(), st, T, tstride, tslice, nx_out,
                    ny_out, out, out_stride, sub, partials, tw, sm);
}

template <typename R, int P>
cudaError_t FftLen<R, P>::row_resid(cx<R>* T, int tstride, int64_t tslice, int nx, int ny, const R* y,
                                    int64_t y_stride, int S, double* partials, double* total,
                                    unsigned* count, const cx<R>* tw, cudaStream_t st, int* nblocks,
                                    Samp sm) {
  using SH = Shape<P>;
  auto fn = sm.on ? k_row_resid<R, P, true> : k_row_resid<R, P, false>;
  const size_t smem =
      smem_bytes<R, P>() + (sm.on ? ResidStage<R, P, true>::bytes : ResidStage<R, P, false>::bytes);
  cudaError_t e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int pairs = (ny + 1) / 2;
  dim3 grid((pairs + SH::VPB - 1) / SH::VPB, S);
  *nblocks = (int)(grid.x * grid.y);
  return launch_pdl(fn, grid, dim3(kThreads), smem, st, T, tstride, tslice, nx, ny, y, y_stride,
                    partials, partials ? total : nullptr, count, tw, sm);
}

template <typename R, int P>
cudaError_t FftLen<R, P>::row_c2r_step(const cx<R>* T, int tstride, int64_t tslice, int nx, int ny,
                                       int64_t plane, int S, const FistaStep& f, const cx<R>* tw,
                                       cudaStream_t st) {
  using SH = Shape<P>;
  auto fn = f.next_T ? k_row_c2r_step<R, P, true> : k_row_c2r_step<R, P, false>;
  const size_t smem = smem_bytes<R, P>() + StepStage<R, P>::bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int pairs = (ny + 1) / 2;
  dim3 grid((pairs + SH::VPB - 1) / SH::VPB, S);
  return launch_pdl(fn, grid, dim3(kThreads), smem, st, const_cast<cx<R>*>(T), tstride,
                    tslice, nx, ny, plane, static_cast<R*>(f.y), static_cast<R*>(f.xprev), f.scal,
                    f.betas, f.iter, f.r2_cur, f.r2_hist, f.cap, f.done, tw);
}

// Explicit instantiation of every launcher for one (precision, length).
#define PAT_FFT_INSTANTIATE(R, P) template struct FftLen<R, P>;

}  // namespace pat
