// Shared-memory Stockham FFT for batches of lines whose length is 2^a 3^b.
//
// The x and z directions of the grid are periodic, so the constant-coefficient
// pressure equation (Eq. (34) of the paper, solved directly by a fast Poisson
// solver as stated after it) is diagonal in the discrete Fourier basis along x
// and z; the y pass uses the same routine inside its cosine transform.  These
// device routines transform many lines at once, held in shared memory by one
// CTA.
//
// One pass of radix R over a line of length n (Stockham autosort, no bit
// reversal): with Ns the product of the radices already applied, butterfly t
// (0 <= t < n/R) reads the R elements t + q n/R, multiplies element q by
// w^(q k n/(Ns R)) with k = t mod Ns and w = exp(-+ 2 pi i / n), takes the
// R-point DFT in registers and writes output q to (t/Ns) Ns R + k + q Ns.
// Passes alternate between two buffers.  Radices 16 and 8 are built from 4x4
// and 2x4 in registers (Cooley-Tukey), so a 256-point line takes two passes.
// Forward transforms use w = exp(-2 pi i/n), inverse ones exp(+2 pi i/n);
// neither is scaled.  Consecutive threads take consecutive lines (the line
// index is the fast one), so twiddle reads are warp broadcasts.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dfloat.cuh"
#include "fastdiv.cuh"

namespace ppe {

// Aligned to its full size, so that one element moves with one 8-byte (FP32) or
// 16-byte (FP64) access.
template <typename T> struct alignas(2 * sizeof(T)) cpx { T x, y; };

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  cpx<T> r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// pairs: each component with one normalisation (dd_dot2)
__device__ __forceinline__ cpx<dd> cmul(cpx<dd> a, cpx<dd> b) {
  return {dd_dot2<true>(a.x, b.x, a.y, b.y), dd_dot2<false>(a.x, b.y, a.y, b.x)};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cpx<T> rot(cpx<T> a) {
  return INV ? cpx<T>{-a.y, a.x} : cpx<T>{a.y, -a.x};
}

// Radices applied in order; n = prod r[s]; ns[s] divides by the product of
// the radices before stage s.
struct RadixPlan {
  int n;
  int nst;
  int r[16];
  FastDiv ns[16];
};

// exp(-+ 2 pi i m / 16) for a compile-time m, times v.  Multiples of a quarter
// turn are exact rotations; the others use cos(pi/8), sin(pi/8), sqrt(1/2).
template <typename T, bool INV, int M16>
__device__ __forceinline__ cpx<T> tw16(cpx<T> v) {
  constexpr int m = ((M16 % 16) + 16) % 16;
  constexpr double C1 = 0.92387953251128675612818318939679;  // cos(pi/8)
  constexpr double S1 = 0.38268343236508977172845998403040;  // sin(pi/8)
  constexpr double H = 0.70710678118654752440084436210485;   // sqrt(1/2)
  // cos(pi m/8), sin(pi m/8)
  constexpr double c = (m == 0) ? 1 : (m == 1) ? C1 : (m == 2) ? H : (m == 3) ? S1 : (m == 4) ? 0
                     : (m == 5) ? -S1 : (m == 6) ? -H : (m == 7) ? -C1 : (m == 8) ? -1 : (m == 9) ? -C1
                     : (m == 10) ? -H : (m == 11) ? -S1 : (m == 12) ? 0 : (m == 13) ? S1 : (m == 14) ? H : C1;
  constexpr double s = (m == 0) ? 0 : (m == 1) ? S1 : (m == 2) ? H : (m == 3) ? C1 : (m == 4) ? 1
                     : (m == 5) ? C1 : (m == 6) ? H : (m == 7) ? S1 : (m == 8) ? 0 : (m == 9) ? -S1
                     : (m == 10) ? -H : (m == 11) ? -C1 : (m == 12) ? -1 : (m == 13) ? -C1 : (m == 14) ? -H : -S1;
  if (m == 0) return v;
  if (m == 8) return {-v.x, -v.y};
  if (m == 4) return rot<T, INV>(v);                 // -i forward
  if (m == 12) return rot<T, !INV>(v);               // +i forward
  constexpr T cr = (T)c, si = INV ? (T)s : (T)(-s);  // w = c - i s (forward)
  if constexpr (std::is_same<T, dd>::value) return {dd_dot2<true>(v.x, cr, v.y, si), dd_dot2<false>(v.x, si, v.y, cr)};
  else return {v.x * cr - v.y * si, v.x * si + v.y * cr};
}

template <typename T, bool INV, int R> struct SmallDft;

template <typename T, bool INV> struct SmallDft<T, INV, 2> {
  static __device__ __forceinline__ void run(cpx<T>* v) {
    cpx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename T, bool INV> struct SmallDft<T, INV, 3> {
  // y1 = v0 - (v1+v2)/2 -+ i (sqrt(3)/2)(v1 - v2), y2 = conjugate rotation
  static __device__ __forceinline__ void run(cpx<T>* v) {
    constexpr T s3 = (T)0.86602540378443864676372317075294;
    cpx<T> t1 = cadd(v[1], v[2]);
    constexpr T half = (T)0.5;
    cpx<T> t2 = {v[0].x - half * t1.x, v[0].y - half * t1.y};
    cpx<T> d = csub(v[1], v[2]);
    cpx<T> t3 = {s3 * d.x, s3 * d.y};
    v[0] = cadd(v[0], t1);
    cpx<T> r = rot<T, INV>(t3);
    v[1] = cadd(t2, r);
    v[2] = csub(t2, r);
  }
};

template <typename T, bool INV> struct SmallDft<T, INV, 4> {
  static __device__ __forceinline__ void run(cpx<T>* v) {
    cpx<T> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    cpx<T> b0 = cadd(v[1], v[3]), b1 = rot<T, INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, b0);
    v[2] = csub(a0, b0);
    v[1] = cadd(a1, b1);
    v[3] = csub(a1, b1);
  }
};

// Pairs: the butterflies' adds are lazy (dd_add_lazy) and each output is
// normalised once at the end, so every value leaving a small DFT is a
// normalised pair (the larger radices are built from these).
__device__ __forceinline__ cpx<dd> cadd_l(cpx<dd> a, cpx<dd> b) { return {dd_add_lazy(a.x, b.x), dd_add_lazy(a.y, b.y)}; }
__device__ __forceinline__ cpx<dd> csub_l(cpx<dd> a, cpx<dd> b) { return {dd_sub_lazy(a.x, b.x), dd_sub_lazy(a.y, b.y)}; }
__device__ __forceinline__ cpx<dd> cnorm(cpx<dd> a) { return {dd_norm(a.x), dd_norm(a.y)}; }

template <bool INV> struct SmallDft<dd, INV, 2> {
  static __device__ __forceinline__ void run(cpx<dd>* v) {
    const cpx<dd> a = v[0], b = v[1];
    v[0] = cnorm(cadd_l(a, b));
    v[1] = cnorm(csub_l(a, b));
  }
};

template <bool INV> struct SmallDft<dd, INV, 3> {
  static __device__ __forceinline__ void run(cpx<dd>* v) {
    constexpr dd s3 = dd(0.86602540378443864676372317075294);
    const cpx<dd> t1 = cadd_l(v[1], v[2]);
    // v0 - t1/2 (halving is exact on both parts)
    const cpx<dd> h = {dd(0.5f * t1.x.hi, 0.5f * t1.x.lo), dd(0.5f * t1.y.hi, 0.5f * t1.y.lo)};
    const cpx<dd> t2 = csub_l(v[0], h);
    const cpx<dd> d = csub_l(v[1], v[2]);
    const cpx<dd> t3 = {s3 * d.x, s3 * d.y};
    const cpx<dd> r = rot<dd, INV>(t3);
    v[0] = cnorm(cadd_l(v[0], t1));
    v[1] = cnorm(cadd_l(t2, r));
    v[2] = cnorm(csub_l(t2, r));
  }
};

template <bool INV> struct SmallDft<dd, INV, 4> {
  static __device__ __forceinline__ void run(cpx<dd>* v) {
    const cpx<dd> a0 = cadd_l(v[0], v[2]), a1 = csub_l(v[0], v[2]);
    const cpx<dd> b0 = cadd_l(v[1], v[3]), b1 = rot<dd, INV>(csub_l(v[1], v[3]));
    v[0] = cnorm(cadd_l(a0, b0));
    v[2] = cnorm(csub_l(a0, b0));
    v[1] = cnorm(cadd_l(a1, b1));
    v[3] = cnorm(csub_l(a1, b1));
  }
};

// R = R1 R2 from an R1-point and an R2-point DFT: sub-DFTs of size R1 on the
// stride-R2 subsequences, twiddles w_R^(j2 k1), then size-R2 DFTs:
// X[k1 + R1 k2] = sum_j2 w_R^(j2 k1) w_R2^(j2 k2) sum_j1 v[j2 + R2 j1] w_R1^(j1 k1).
template <typename T, bool INV, int R1, int R2>
__device__ __forceinline__ void dft_ct(cpx<T>* v) {
  constexpr int R = R1 * R2;
  cpx<T> a[R];
#pragma unroll
  for (int j2 = 0; j2 < R2; ++j2) {
    cpx<T> s[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) s[j1] = v[j2 + R2 * j1];
    SmallDft<T, INV, R1>::run(s);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[j2 * R1 + k1] = s[k1];
  }
  // twiddles w_R^(j2 k1) = w_16^(j2 k1 16/R)
#pragma unroll
  for (int j2 = 1; j2 < R2; ++j2) {
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      cpx<T>& x = a[j2 * R1 + k1];
      const int e = j2 * k1 * (16 / R);
      switch (e) {  // resolved at compile time after unrolling
        case 1: x = tw16<T, INV, 1>(x); break;
        case 2: x = tw16<T, INV, 2>(x); break;
        case 3: x = tw16<T, INV, 3>(x); break;
        case 4: x = tw16<T, INV, 4>(x); break;
        case 6: x = tw16<T, INV, 6>(x); break;
        case 8: x = tw16<T, INV, 8>(x); break;
        case 9: x = tw16<T, INV, 9>(x); break;
        case 12: x = tw16<T, INV, 12>(x); break;
        default: break;
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    cpx<T> s[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) s[j2] = a[j2 * R1 + k1];
    SmallDft<T, INV, R2>::run(s);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = s[k2];
  }
}

template <typename T, bool INV> struct SmallDft<T, INV, 8> {
  static __device__ __forceinline__ void run(cpx<T>* v) { dft_ct<T, INV, 2, 4>(v); }
};
template <typename T, bool INV> struct SmallDft<T, INV, 16> {
  static __device__ __forceinline__ void run(cpx<T>* v) { dft_ct<T, INV, 4, 4>(v); }
};

// One Stockham pass over nl = 2^nl_log2 lines (nl <= blockDim.x, blockDim.x a
// power of two).  Line `l`, element `e` lives at base[l*ls + e*es].
// Consecutive threads take consecutive lines.  `tw` (shared memory) holds
// exp(-2 pi i t / (n*tws)), t < n*tws.
template <typename T, bool INV, int R>
__device__ __forceinline__ void stockham_pass(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst, int nl_log2,
                                              int n, int ls, int es, int Ns, const FastDiv& nsdiv,
                                              const cpx<T>* __restrict__ tw, int tws) {
  const int nb = n / R;
  const int tstep = n / (Ns * R);
  const int line = threadIdx.x & ((1 << nl_log2) - 1);
  const int t0 = threadIdx.x >> nl_log2, ts = blockDim.x >> nl_log2;
  const cpx<T>* s = src + line * ls;
  cpx<T>* d = dst + line * ls;
  for (int t = t0; t < nb; t += ts) {
    const int q0 = (int)fdiv((uint32_t)t, nsdiv);
    const int k = t - q0 * Ns;
    cpx<T> v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = s[(t + q * nb) * es];
    if (Ns > 1) {
      const int e1 = tstep * k * tws;
#pragma unroll
      for (int q = 1; q < R; ++q) {
        cpx<T> w = tw[q * e1];
        if (INV) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    SmallDft<T, INV, R>::run(v);
    const int base = q0 * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) d[(base + q * Ns) * es] = v[q];
  }
}

// Full transform of 2^nl_log2 lines held in `a` (with `b` as the second
// buffer).  The caller synchronises before the call; the routine synchronises
// after every pass and returns the buffer that holds the result.
template <typename T, bool INV>
__device__ cpx<T>* fft_lines(cpx<T>* a, cpx<T>* b, int nl_log2, const RadixPlan& rp, int ls, int es,
                             const cpx<T>* __restrict__ tw, int tws) {
  int Ns = 1;
  for (int s = 0; s < rp.nst; ++s) {
    const int R = rp.r[s];
    switch (R) {
      case 16: stockham_pass<T, INV, 16>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws); break;
      case 8: stockham_pass<T, INV, 8>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws); break;
      case 4: stockham_pass<T, INV, 4>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws); break;
      case 2: stockham_pass<T, INV, 2>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws); break;
      default: stockham_pass<T, INV, 3>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws); break;
    }
    __syncthreads();
    cpx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// ---------------------------------------------------------------------------
// Compile-time-length variant.  With n, the radices, Ns and n/R known to the
// compiler, every per-element index and twiddle offset becomes an immediate or
// one multiply-add, and the butterfly loop bounds are constants.  Same passes
// and results as fft_lines; used for the lengths of the common grids.
// ---------------------------------------------------------------------------
namespace ctfft {

// The radix sequence of radix_plan() (host): radix 16 while it divides (if
// maxr >= 16), one 8 (if maxr >= 8), 4s, one 2, then 3s.
__host__ __device__ constexpr int radix_at(int n, int s, int maxr) {
  int m = n, i = 0;
  while (maxr >= 16 && m % 16 == 0) { if (i == s) return 16; m /= 16; ++i; }
  if (maxr >= 8 && m % 8 == 0) { if (i == s) return 8; m /= 8; ++i; }
  while (m % 4 == 0) { if (i == s) return 4; m /= 4; ++i; }
  if (m % 2 == 0) { if (i == s) return 2; m /= 2; ++i; }
  while (m % 3 == 0) { if (i == s) return 3; m /= 3; ++i; }
  return 1;
}
__host__ __device__ constexpr int nst(int n, int maxr) {
  int s = 0;
  while (radix_at(n, s, maxr) != 1) ++s;
  return s;
}
__host__ __device__ constexpr int ns_at(int n, int s, int maxr) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= radix_at(n, i, maxr);
  return p;
}

template <typename T, bool INV, int N, int S, int MAXR, int TWS>
__device__ __forceinline__ void pass_ct(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst, int nl_log2,
                                        int ls, int es, const cpx<T>* __restrict__ tw) {
  constexpr int R = radix_at(N, S, MAXR);
  constexpr int NS = ns_at(N, S, MAXR);
  constexpr int NB = N / R;
  constexpr int TSTEP = N / (NS * R);
  const int line = threadIdx.x & ((1 << nl_log2) - 1);
  const int t0 = threadIdx.x >> nl_log2, ts = blockDim.x >> nl_log2;
  const cpx<T>* s = src + line * ls;
  cpx<T>* d = dst + line * ls;
  const int sb = NB * es, sq = NS * es;
  for (int t = t0; t < NB; t += ts) {
    const int q0 = t / NS, k = t - q0 * NS;  // NS a power of 2 times 3^b, known here
    cpx<T> v[R];
    const cpx<T>* sp = s + t * es;
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = sp[q * sb];
    if (NS > 1) {
      const int e1 = TSTEP * TWS * k;
#pragma unroll
      for (int q = 1; q < R; ++q) {
        cpx<T> w = tw[q * e1];
        if (INV) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    SmallDft<T, INV, R>::run(v);
    cpx<T>* dp = d + (q0 * NS * R + k) * es;
#pragma unroll
    for (int q = 0; q < R; ++q) dp[q * sq] = v[q];
  }
}

template <typename T, bool INV, int N, int S, int MAXR, int TWS>
__device__ __forceinline__ cpx<T>* run_from(cpx<T>* a, cpx<T>* b, int nl_log2, int ls, int es,
                                            const cpx<T>* __restrict__ tw) {
  if constexpr (S >= nst(N, MAXR)) {
    return a;
  } else {
    pass_ct<T, INV, N, S, MAXR, TWS>(a, b, nl_log2, ls, es, tw);
    __syncthreads();
    return run_from<T, INV, N, S + 1, MAXR, TWS>(b, a, nl_log2, ls, es, tw);
  }
}

}  // namespace ctfft

// fft_lines for a compile-time length N (radices up to MAXR, twiddle stride TWS)
template <typename T, bool INV, int N, int MAXR, int TWS>
__device__ __forceinline__ cpx<T>* fft_lines_ct(cpx<T>* a, cpx<T>* b, int nl_log2, int ls, int es,
                                                const cpx<T>* __restrict__ tw) {
  return ctfft::run_from<T, INV, N, 0, MAXR, TWS>(a, b, nl_log2, ls, es, tw);
}


// ---------------------------------------------------------------------------
// Register-staged variant for power-of-two lengths 16 <= N <= 512 (FP32
// lines).  Each line is transformed by TPL = N/16 threads; between passes a
// thread keeps 16 elements in registers, so a pass costs one shared-memory
// store and one load per element, and there is no separate staging copy: the
// first pass takes its butterfly inputs from a caller functor `ld(e)` (global
// memory, values computed on the fly, or the shared buffer) and the last pass
// hands its outputs to `st(e, v)`.  Radix sequence, twiddles and butterflies
// are those of fft_lines_ct.
//
// Shared layout: element e of the thread's line at ln[row(e) * es], ln the
// line's base; row(e) = e + e/16 inserts one padding row every 16 elements,
// so that the strided writes of the first pass (rows 16 t + q for the t of a
// warp) fall on different banks.  Lines across columns (z and y passes: lines
// fastest, es = lines per CTA) or along rows (x passes: es = 1, line stride
// chosen by the caller).
// ---------------------------------------------------------------------------
namespace rgfft {

__host__ __device__ constexpr int rows(int n) { return n + n / 16; }
__device__ __forceinline__ int row(int e) { return e + (e >> 4); }
// Position of element e in a line, by layout:
//   PAD_ROWS (true):  row(e), one padding row every 16 elements;
//   DENSE (false):    e (a buffer laid out by a bulk copy whose lines run across
//                     columns, so that a warp's lanes touch consecutive words);
//   XOR_ROWS (2):     e ^ ((e >> 4) & 15), a permutation within each group of
//                     16 that needs no extra space: a line stored along a dense
//                     row (bulk-copied) with its M/16 threads as consecutive
//                     lanes reads and writes 16 distinct 8-byte bank slots in
//                     both Stockham index patterns (16 t + q and t + 16 q).
enum RowLayout { DENSE = 0, PAD_ROWS = 1, XOR_ROWS = 2 };
template <int LAYOUT>
__device__ __forceinline__ int rowp(int e) {
  return LAYOUT == PAD_ROWS ? row(e) : (LAYOUT == XOR_ROWS ? (e ^ ((e >> 4) & 15)) : e);
}

// LD_SHARED: ld reads the shared buffer (the first pass then waits for all
// reads before writing); later passes always read all before their stores.
template <typename T, bool INV, int N, int S, int TWS, bool LD_SHARED, int PAD, class Ld, class St>
__device__ __forceinline__ void pass(Ld& ld, St& st, cpx<T>* ln, int es, int t0, const cpx<T>* __restrict__ tw) {
  using namespace ctfft;
  constexpr int NST = nst(N, 16);
  constexpr int R = radix_at(N, S, 16);
  constexpr int NS = ns_at(N, S, 16);
  constexpr int NB = N / R;
  constexpr int TPL = N / 16;
  constexpr int IT = NB / TPL;
  constexpr int TSTEP = N / (NS * R);
  static_assert(IT * R == 16, "a thread holds 16 elements per pass");
  cpx<T> v[IT][R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int t = t0 + it * TPL;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int e = t + q * NB;
      if (S == 0) v[it][q] = ld(e);
      else v[it][q] = ln[rowp<PAD>(e) * es];
    }
  }
  if (S > 0 || LD_SHARED) __syncthreads();  // in place: every read of the pass before any write
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int t = t0 + it * TPL;
    const int q0 = t / NS, k = t - q0 * NS;
    if (NS > 1) {
      const int e1 = TSTEP * TWS * k;
#pragma unroll
      for (int q = 1; q < R; ++q) {
        cpx<T> w = tw[q * e1];
        if (INV) w.y = -w.y;
        v[it][q] = cmul(v[it][q], w);
      }
    }
    SmallDft<T, INV, R>::run(v[it]);
    const int o = q0 * NS * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (S + 1 == NST) st(o + q * NS, v[it][q]);
      else ln[rowp<PAD>(o + q * NS) * es] = v[it][q];
    }
  }
  if (S + 1 < NST) __syncthreads();
}

template <typename T, bool INV, int N, int S, int TWS, bool LD_SHARED, int PAD, class Ld, class St>
__device__ __forceinline__ void run_from(Ld& ld, St& st, cpx<T>* ln, int es, int t0, const cpx<T>* __restrict__ tw) {
  if constexpr (S < ctfft::nst(N, 16)) {
    pass<T, INV, N, S, TWS, LD_SHARED, PAD>(ld, st, ln, es, t0, tw);
    run_from<T, INV, N, S + 1, TWS, LD_SHARED, PAD>(ld, st, ln, es, t0, tw);
  }
}

// Transform of the CTA's lines (N/16 threads per line, every thread of the
// CTA calls; t0 in [0, N/16) is the thread's rank within its line).  `tw`
// holds exp(-2 pi i t/(N*TWS)) and must be visible to all threads before the
// second pass (the barrier after the first pass suffices when it is written
// before the call).  The caller synchronises after the call before reusing
// the buffer.
template <typename T, bool INV, int N, int TWS, bool LD_SHARED, int PAD = PAD_ROWS, class Ld, class St>
__device__ __forceinline__ void run(Ld&& ld, St&& st, cpx<T>* ln, int es, int t0, const cpx<T>* __restrict__ tw) {
  static_assert((N & (N - 1)) == 0 && N >= 16 && N <= 512, "power-of-two length");
  run_from<T, INV, N, 0, TWS, LD_SHARED, PAD>(ld, st, ln, es, t0, tw);
}

template <int N> struct is_rg : std::integral_constant<bool, (N >= 16 && N <= 512 && (N & (N - 1)) == 0)> {};

}  // namespace rgfft

}  // namespace ppe
