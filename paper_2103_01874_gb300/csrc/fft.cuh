// Shared-memory Stockham FFT for batches of lines whose length is 2^a 3^b.
//
// The x and z directions of the grid are periodic, so the constant-coefficient
// pressure equation (Eq. (34) of the paper, solved directly by a fast Poisson
// solver as stated after it) is diagonal in the discrete Fourier basis along x
// and z.  These device routines transform many such lines at once, the lines
// held in shared memory by one CTA.
//
// One pass of radix R over a line of length n (Stockham autosort, so no bit
// reversal): with Ns the product of the radices already applied, butterfly t
// (0 <= t < n/R) reads the R elements t + q n/R, multiplies element q by
// w^(q k n/(Ns R)) with k = t mod Ns and w = exp(-+ 2 pi i / n), takes the
// R-point DFT and writes output q to (t/Ns) Ns R + k + q Ns.  Passes alternate
// between two buffers.  Forward transforms use w = exp(-2 pi i/n), inverse
// ones exp(+2 pi i/n); neither is scaled.
#pragma once
#include <cuda_runtime.h>

#include "fastdiv.cuh"

namespace ppe {

template <typename T> struct cpx { T x, y; };

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  cpx<T> r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
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
    const T s3 = (T)0.86602540378443864676372317075294;
    cpx<T> t1 = cadd(v[1], v[2]);
    cpx<T> t2 = {v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y};
    cpx<T> d = csub(v[1], v[2]);
    cpx<T> t3 = {s3 * d.x, s3 * d.y};
    v[0] = cadd(v[0], t1);
    cpx<T> r = rot<T, INV>(t3);  // -i t3 forward
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

// One Stockham pass over nl = 2^nl_log2 lines (nl <= blockDim.x, blockDim.x a
// power of two).  Line `l`, element `e` lives at base[l*ls + e*es].  With
// line_fastest, consecutive threads take consecutive lines (suits lines that
// are interleaved in memory, es > 1); otherwise each line gets blockDim/nl
// consecutive threads.  No integer division: shifts, masks and a
// multiply-high divider for Ns.
template <typename T, bool INV, int R>
__device__ __forceinline__ void stockham_pass(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst, int nl_log2,
                                              int n, int ls, int es, int Ns, const FastDiv& nsdiv,
                                              const cpx<T>* __restrict__ tw, int tws, bool line_fastest) {
  const int nb = n / R;
  const int tstep = n / (Ns * R);
  const int bl = __ffs(blockDim.x) - 1;
  int line, t0, ts;
  if (line_fastest) {
    line = threadIdx.x & ((1 << nl_log2) - 1);
    t0 = threadIdx.x >> nl_log2;
    ts = blockDim.x >> nl_log2;
  } else {
    const int tl = bl - nl_log2;  // log2 threads per line
    line = threadIdx.x >> tl;
    t0 = threadIdx.x & ((1 << tl) - 1);
    ts = 1 << tl;
  }
  const cpx<T>* s = src + line * ls;
  cpx<T>* d = dst + line * ls;
  for (int t = t0; t < nb; t += ts) {
    const int q0 = (int)fdiv((uint32_t)t, nsdiv);
    const int k = t - q0 * Ns;
    cpx<T> v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = s[(t + q * nb) * es];
    if (Ns > 1) {
      const int e1 = tstep * k;
#pragma unroll
      for (int q = 1; q < R; ++q) {
        cpx<T> w = tw[(q * e1) * tws];
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
// after every pass and returns the buffer that holds the result.  `tw` is the
// table exp(-2 pi i t / (n*tws)), t < n*tws.
template <typename T, bool INV>
__device__ cpx<T>* fft_lines(cpx<T>* a, cpx<T>* b, int nl_log2, const RadixPlan& rp, int ls, int es,
                             const cpx<T>* __restrict__ tw, int tws, bool line_fastest) {
  int Ns = 1;
  for (int s = 0; s < rp.nst; ++s) {
    const int R = rp.r[s];
    if (R == 4)
      stockham_pass<T, INV, 4>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws, line_fastest);
    else if (R == 2)
      stockham_pass<T, INV, 2>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws, line_fastest);
    else
      stockham_pass<T, INV, 3>(a, b, nl_log2, rp.n, ls, es, Ns, rp.ns[s], tw, tws, line_fastest);
    __syncthreads();
    cpx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

}  // namespace ppe
