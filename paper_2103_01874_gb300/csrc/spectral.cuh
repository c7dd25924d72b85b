// Spectral kernels of the direct Poisson solve of Eq. (34) (the fast Poisson
// solver stated after Eq. (34): periodic x and z, homogeneous Neumann walls in y).
// Templates on the element type T, instantiated for FP32 (k_spectral_f32.cu,
// with the register-staged forms), FP64 (k_spectral_f64.cu) and double-float
// pairs dd (k_spectral_dd.cu), one translation unit each so that they build in
// parallel.
//
// Spectrum layout (plan workspace): complex T, [kz][j][kx] with kx fastest,
// kx = 0 .. nx/2 (nxh = nx/2 + 1 values, the real-input half spectrum), j the
// physical wall-normal index, kz = 0 .. nz-1.  Every pass works in place.
//
//   k_xfwd    one CTA per `lpb` x-lines: builds the real line (a given f, or
//             the residual f - L p of the refinement in pair arithmetic), packs
//             it as nx/2 complex values, FFTs them and untangles the nx/2+1
//             half spectrum.  (The Eq. (34) right-hand side has its own fused
//             kernel, k_rhs.cu.)
//   k_zfft    one CTA per (j, tile of `tkx` kx columns): FFT along z.
//   k_ythomas one thread per (kx, kz): the Neumann tridiagonal solve in y with
//             precomputed elimination multipliers; zero mode pinned.
//   k_xinv    one CTA per `lpb` lines: half spectrum -> real line, scaled, and
//             stored to p (FP64), stored as pairs, or added to the pairs
//             (refinement update).
#pragma once
#include <type_traits>

#include "async.cuh"
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "pdl.cuh"
#include "stencil.cuh"

namespace ppe {

template <typename T>
__device__ __forceinline__ cpx<T> ld_tw(const cpx<T>* tw, int t) {
  return tw[t];
}

// log2 of a power of two
__device__ __forceinline__ int ilog2_dev(int v) { return __ffs(v) - 1; }

// FP32 and pair passes have compile-time-length instances (register-staged
// for powers of two); FP64 passes run on run-time radix plans
template <typename T>
struct has_ct_lengths : std::integral_constant<bool, sizeof(T) == 4 || std::is_same<T, dd>::value> {};

// Transform with the compile-time-length passes when N > 0 (FP32 and pair
// lengths; radices up to 16 in FP32 and 8 in pairs, which measured faster at
// their register counts), else with the run-time-length ones (as radix_plan()).
template <typename T, bool INV, int N, int TWS>
__device__ __forceinline__ cpx<T>* fft_any(cpx<T>* a, cpx<T>* b, int nl_log2, const RadixPlan& rp, int ls, int es,
                                          const cpx<T>* __restrict__ tw) {
  if constexpr (N > 0) {
    return fft_lines_ct<T, INV, N, (sizeof(T) == 4 ? 16 : 8), TWS>(a, b, nl_log2, ls, es, tw);
  } else {
    return fft_lines<T, INV>(a, b, nl_log2, rp, ls, es, tw, TWS);
  }
}

// Calls f(std::integral_constant<int, N>) with N = n for the lengths that have
// compile-time instances (FP32 only), N = 0 otherwise.
// reciprocal for the eigenvalue divide: the correctly rounded float reciprocal,
// or the pair reciprocal
template <typename T>
__device__ __forceinline__ T rcp_of(T x) {
  if constexpr (std::is_same<T, dd>::value) return dd(df_recip(x.pair()));
  else return __frcp_rn(x);
}


template <typename T, typename F>
cudaError_t with_len(int n, F&& f) {
  if constexpr (has_ct_lengths<T>::value) {
    switch (n) {
      case 16: return f(std::integral_constant<int, 16>{});
      case 24: return f(std::integral_constant<int, 24>{});
      case 32: return f(std::integral_constant<int, 32>{});
      case 48: return f(std::integral_constant<int, 48>{});
      case 64: return f(std::integral_constant<int, 64>{});
      case 96: return f(std::integral_constant<int, 96>{});
      case 128: return f(std::integral_constant<int, 128>{});
      case 192: return f(std::integral_constant<int, 192>{});
      case 256: return f(std::integral_constant<int, 256>{});
      case 384: return f(std::integral_constant<int, 384>{});
      default: break;
    }
  }
  return f(std::integral_constant<int, 0>{});
}

// Kernels needing more than the default 48 KB of dynamic shared memory opt in.
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------------
// forward x pass
// ---------------------------------------------------------------------------
// OPEN: the residual's top cells see the outflow ghost (SRC_RESID only)
template <typename T, int SRC, bool DO_FFT, int N, bool OPEN = false>
__device__ __forceinline__ void xfwd_body(GridDev g, StencilIn in, DevScalars* sc, int slot, df* fdf,
                                              const df* pdf, cpx<T>* spec, RadixPlan rp,
                                              const cpx<T>* tw, int lpb, uint32_t bid, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (SRC == SRC_RESID && slot < 0) slot = sc->iter;  // residual slot chosen on the device
  const int nx = g.nx, M = nx / 2, nxh = M + 1;
  const int lsc = M + 1;  // padded line stride (complex elements) against bank conflicts
  const int nlines = g.ny * g.nz;
  const int l0 = bid * lpb;
  cpx<T>* bufa = reinterpret_cast<cpx<T>*>(smem_raw);  // lpb lines of lsc; line ll holds its nx reals packed
  cpx<T>* bufb = bufa + (size_t)lpb * lsc;
  cpx<T>* tws = bufb + (size_t)lpb * lsc;           // twiddles exp(-2 pi i t/nx), t < nx
  T* line_re = reinterpret_cast<T*>(bufa);
  if (DO_FFT) {
    for (int t = threadIdx.x; t < nx; t += blockDim.x) cp_async<sizeof(cpx<T>)>(&tws[t], &tw[t]);
  }

  df lc[3];
  if (SRC == SRC_RESID) {
    lc[0] = sc->K.lx;
    lc[1] = sc->K.ly;
    lc[2] = sc->K.lz;
  }
  float vmax = 0.0f;
  df fmean = {0.0f, 0.0f};  // SRC_RESID: mean of f, left out of the residual (the solve drops it)
  if (SRC == SRC_RESID) fmean = sc->f_mean;
  df fsum = {0.0f, 0.0f};  // SRC_F / SRC_FDF: sum of f over this thread's cells
  if (SRC == SRC_F) {
    for (int idx = threadIdx.x; idx < lpb * nx; idx += blockDim.x) {
      const int ll = (int)fdiv(idx, g.fd_nx);
      const int line = l0 + ll;
      T val = (T)0;
      if (line < nlines) {
        const size_t c = (size_t)l0 * nx + idx;
        const double x = __ldg(in.f + c);
        const df v = d2df(x);
        if constexpr (std::is_same<T, dd>::value) {
          val = T(v);
        } else if constexpr (sizeof(T) == 8) {
          val = (T)x;
        } else {
          if (fdf) fdf[c] = v;
          val = (T)df_to_f(v);
        }
        vmax = fmaxf(vmax, fabsf(v.hi));
        fsum = df_addz(fsum, v);
      }
      line_re[idx + ll * 2] = val;  // line ll starts at 2*ll*lsc = ll*nx + 2*ll
    }
  } else if (SRC == SRC_FDF) {
    // f as pairs, written by the right-hand-side kernel (which also took ||f||);
    // four loads per thread in flight before the first use
    constexpr int U = 4;
    for (int b0 = 0; b0 < lpb * nx; b0 += U * blockDim.x) {
      df v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * blockDim.x + threadIdx.x;
        const int ll = (int)fdiv(idx, g.fd_nx);
        v[u] = (idx < lpb * nx && l0 + ll < nlines) ? fdf[(size_t)l0 * nx + idx] : df{0.0f, 0.0f};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * blockDim.x + threadIdx.x;
        if (idx >= lpb * nx) continue;
        const int ll = (int)fdiv(idx, g.fd_nx);
        if constexpr (std::is_same<T, dd>::value) line_re[idx + ll * 2] = T(v[u]);
        else line_re[idx + ll * 2] = (sizeof(T) == 8) ? (T)df2d_alu(v[u]) : (T)df_to_f(v[u]);
        fsum = df_addz(fsum, v[u]);
      }
    }
  } else {
    // residual r = f - L p in pairs; two cells per thread per round with all
    // their loads issued first
    constexpr int U = 2;
    for (int b0 = 0; b0 < lpb * nx; b0 += U * blockDim.x) {
      df pc[U], pxp[U], pxm[U], pyp[U], pym[U], pzp[U], pzm[U], fv[U];
      int jj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * blockDim.x + threadIdx.x;
        const int ll = (int)fdiv(idx, g.fd_nx), i = idx - ll * nx;
        const int line = l0 + ll;
        jj[u] = -1;
        if (idx < lpb * nx && line < nlines) {
          // 32-bit offsets (grids up to 1024^3)
          const uint32_t k = fdiv((uint32_t)line, g.fd_ny), j = (uint32_t)line - k * (uint32_t)g.ny;
          const uint32_t plane = (uint32_t)g.ny * (uint32_t)nx, nzu = (uint32_t)g.nz;
          const uint32_t c = (uint32_t)line * (uint32_t)nx + (uint32_t)i;
          jj[u] = (int)j;
          pc[u] = pdf[c];
          pxp[u] = pdf[(i + 1 == nx) ? c + 1 - nx : c + 1];
          pxm[u] = pdf[(i == 0) ? c + nx - 1 : c - 1];
          pzp[u] = pdf[(k + 1 == nzu) ? c - (nzu - 1) * plane : c + plane];
          pzm[u] = pdf[(k == 0) ? c + (nzu - 1) * plane : c - plane];
          // above the top cell: the wall mirror, or the outflow ghost -p (p = 0 on the face)
          pyp[u] = (j + 1 < (uint32_t)g.ny) ? pdf[c + nx] : (OPEN ? df_neg(pc[u]) : pc[u]);
          pym[u] = (j > 0) ? pdf[c - nx] : pc[u];
          fv[u] = fdf[c];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * blockDim.x + threadIdx.x;
        if (idx >= lpb * nx) continue;
        T val = (T)0;
        if (jj[u] >= 0) {
          // second differences as (p+ + p-) - 2 p (the wall sides contribute 0)
          const df p2 = df_ldexp2(pc[u]);
          const df lx = df_subz(df_addz(pxp[u], pxm[u]), p2);
          const df lz = df_subz(df_addz(pzp[u], pzm[u]), p2);
          const df ly = df_subz(df_addz(pyp[u], pym[u]), p2);
          const df lap = df_addz(df_addz(df_mulz(lx, lc[0]), df_mulz(ly, lc[1])), df_mulz(lz, lc[2]));
          const float r = df_to_f(df_subz(df_subz(fv[u], fmean), lap));
          val = T(r);
          vmax = fmaxf(vmax, fabsf(r));
        }
        line_re[idx + (int)fdiv(idx, g.fd_nx) * 2] = val;
      }
    }
  }
  if (SRC == SRC_F) block_max_to(&sc->fmax_bits, vmax);
  else if (SRC == SRC_RESID) block_max_to(&sc->rmax_bits[slot], vmax);  // float max, widened once per warp
  if (SRC == SRC_F || SRC == SRC_FDF) {
    // per-CTA sum of f, totalled in a fixed order by the next kernel (finish_sums)
    block_pair_sums(fsum, df{0.0f, 0.0f}, sc->part + (size_t)g.ny * g.nz + bid);
    if (bid == 0 && threadIdx.x == 0) sc->x_parts = (int)nblk;
  }
  if (!DO_FFT) return;
  cp_async_wait_all();
  __syncthreads();
  cpx<T>* z = fft_any<T, false, N, 2>(bufa, bufb, ilog2_dev(lpb), rp, lsc, 1, tws);
  // untangle: X_k = (Z_k + conj Z_{M-k})/2 - i W^k (Z_k - conj Z_{M-k})/2, W = exp(-2 pi i/nx)
  for (int idx = threadIdx.x; idx < lpb * nxh; idx += blockDim.x) {
    const int ll = (int)fdiv(idx, g.fd_nxh), kx = idx - ll * nxh;
    const int line = l0 + ll;
    if (line >= nlines) continue;
    const cpx<T> zk = z[ll * lsc + (kx == M ? 0 : kx)];
    const cpx<T> zc = z[ll * lsc + (kx == 0 ? 0 : M - kx)];
    const cpx<T> a = {zk.x + zc.x, zk.y - zc.y};
    const cpx<T> b = {zk.x - zc.x, zk.y + zc.y};
    const cpx<T> wb = cmul(tws[kx], b);
    cpx<T> X;
    X.x = (T)0.5 * (a.x + wb.y);
    X.y = (T)0.5 * (a.y - wb.x);
    spec[(size_t)line * nxh + kx] = X;
  }
}
template <typename T, int SRC, bool DO_FFT, int N, bool OPEN = false>
__global__ void __launch_bounds__(256) k_xfwd(GridDev g, StencilIn in, DevScalars* sc, int slot, df* fdf,
                                              const df* __restrict__ pdf, cpx<T>* spec, RadixPlan rp,
                                              const cpx<T>* __restrict__ tw, int lpb) {
  xfwd_body<T, SRC, DO_FFT, N, OPEN>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb, blockIdx.x, gridDim.x);
}

// Line stride (complex elements) of the x passes' shared buffer: rgfft rows,
// padded to 8 mod 16 so that neighbouring lines start half a bank row apart.
__host__ __device__ constexpr int xrg_stride(int m) { return rgfft::rows(m) + ((8 - rgfft::rows(m) % 16) + 16) % 16; }
// The same for the plane layout of the spectrum (PL): one more element (the
// inverse pass stages X_M too) and padded to 4 mod 16, so that both the FFT
// passes (lanes: 32/(M/16) lines of M/16 threads) and the transposing copies
// (lanes: 8 lines x 4 kx) touch each 8-byte bank slot at most twice per warp.
__host__ __device__ constexpr int xrg_stride_pl(int m) {
  return (rgfft::rows(m) + 1) + ((4 - (rgfft::rows(m) + 1) % 16) + 16) % 16;
}
template <bool PL>
__host__ __device__ constexpr int xstride(int m) { return PL ? xrg_stride_pl(m) : xrg_stride(m); }

// Lane split of the transposing copies of the plane layout: LQ consecutive
// lines (8, or all L when fewer) times 32/LQ consecutive kx per warp, so that a
// warp moves 64-byte runs of one kx plane.
struct PlaneLanes {
  int lq, kq;
};
__device__ __forceinline__ PlaneLanes plane_lanes(int L) { return {L < 8 ? L : 8, 32 / (L < 8 ? L : 8)}; }

// Register-staged forward x pass (FP32, nx = 2M, M a power of two; rgfft in
// fft.cuh).  A CTA of L * M/16 threads owns L consecutive x-lines; thread
// (line, t) forms the packed values z_e = x_{2e} + i x_{2e+1} of its first
// FFT pass (e = t + q M/16) straight from the source -- f (FP64), f as pairs,
// or the residual f - L p in pair arithmetic, two cells per 16-byte load --
// the last pass leaves Z in shared memory and the untangle writes the nx/2 + 1
// half spectrum.  Same cell arithmetic as k_xfwd.
// PL: the spectrum in the plane layout [kx][line] (GridDev::spec_planes).
template <int SRC, int M, bool OPEN, bool PL = false>
__device__ __forceinline__ void xfwd_rg_body(GridDev g, StencilIn in, DevScalars* sc, int slot, df* fdf,
                                                 const df* pdf, cpx<float>* spec,
                                                 const cpx<float>* tw, int L, uint32_t bid, uint32_t nblk) {
  using T = float;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (SRC == SRC_RESID && slot < 0) slot = sc->iter;  // residual slot chosen on the device
  constexpr int TPL = M / 16, nx = 2 * M, nxh = M + 1, LS = xstride<PL>(M);
  const uint32_t nlines = (uint32_t)g.ny * (uint32_t)g.nz;
  const int ll = (int)threadIdx.x / TPL, t0 = (int)threadIdx.x & (TPL - 1);
  const uint32_t l0 = bid * (uint32_t)L;
  const uint32_t line = l0 + ll;
  const bool valid = line < nlines;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);  // L lines of LS
  cpx<T>* tws = buf + L * LS;                          // exp(-2 pi i t/nx), t < nx
  for (int t = threadIdx.x; t < nx; t += blockDim.x) tws[t] = tw[t];
  const uint32_t c0 = line * (uint32_t)nx;  // 32-bit offsets (grids up to 1024^3)
  float vmax = 0.0f;
  df fsum = {0.0f, 0.0f};
  auto put = [&](int e, cpx<T> v) { buf[ll * LS + rgfft::row(e)] = v; };
  if constexpr (SRC == SRC_F) {
    const double2* fl = reinterpret_cast<const double2*>(in.f + c0);
    float4* fo = fdf ? reinterpret_cast<float4*>(fdf + c0) : nullptr;
    // a caller's f off a 16-byte boundary is read with 8-byte loads (the plane
    // layout has no other forward pass to fall back to)
    const bool f16 = !PL || ((uintptr_t)in.f & 15u) == 0;
    rgfft::run<T, false, M, 2, false>(
        [&](int e) -> cpx<T> {
          if (!valid) return {(T)0, (T)0};
          const double2 x = f16 ? __ldg(fl + e) : make_double2(__ldg(in.f + c0 + 2 * e), __ldg(in.f + c0 + 2 * e + 1));
          const df v0 = d2df(x.x), v1 = d2df(x.y);
          if (fo) fo[e] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
          vmax = fmaxf(vmax, fmaxf(fabsf(v0.hi), fabsf(v1.hi)));
          fsum = df_addz(df_addz(fsum, v0), v1);
          return {df_to_f(v0), df_to_f(v1)};
        },
        put, buf + ll * LS, 1, t0, tws);
  } else if constexpr (SRC == SRC_FDF) {
    // f as pairs, written by the right-hand-side kernel (which also took ||f||)
    const float4* fl = reinterpret_cast<const float4*>(fdf + c0);
    rgfft::run<T, false, M, 2, false>(
        [&](int e) -> cpx<T> {
          if (!valid) return {(T)0, (T)0};
          const float4 q = fl[e];
          const df v0 = {q.x, q.y}, v1 = {q.z, q.w};
          fsum = df_addz(df_addz(fsum, v0), v1);
          return {df_to_f(v0), df_to_f(v1)};
        },
        put, buf + ll * LS, 1, t0, tws);
  } else {
    // residual r = f - L p in pairs, second differences as (p+ + p-) - 2 p
    const df lcx = sc->K.lx, lcy = sc->K.ly, lcz = sc->K.lz;
    const df fmean = sc->f_mean;  // left out of the residual (the solve drops it)
    const uint32_t ny = (uint32_t)g.ny, nzu = (uint32_t)g.nz;
    const uint32_t k = valid ? fdiv(line, g.fd_ny) : 0u, j = line - k * ny;
    const uint32_t plane = ny * (uint32_t)nx;
    const df* pl = pdf + c0;
    const float4* pc4 = reinterpret_cast<const float4*>(pl);
    const float4* pzm4 = reinterpret_cast<const float4*>(pdf + (k == 0 ? c0 + (nzu - 1) * plane : c0 - plane));
    const float4* pzp4 = reinterpret_cast<const float4*>(pdf + (k + 1 == nzu ? c0 - (nzu - 1) * plane : c0 + plane));
    const bool has_ym = j > 0, has_yp = j + 1 < ny;
    const float4* pym4 = reinterpret_cast<const float4*>(pdf + (has_ym ? c0 - nx : c0));
    const float4* pyp4 = reinterpret_cast<const float4*>(pdf + (has_yp ? c0 + nx : c0));
    const float4* f4 = reinterpret_cast<const float4*>(fdf + c0);
    // the first sweep may read the first solve's p in FP32 (a pair with a zero
    // low part: the same values)
    const bool p0f = in.p0f != nullptr && sc->iter == 1;
    const float* ql = p0f ? in.p0f + c0 : nullptr;
    const float2* qc2 = reinterpret_cast<const float2*>(ql);
    const float2* qzm2 = reinterpret_cast<const float2*>(p0f ? in.p0f + (k == 0 ? c0 + (nzu - 1) * plane : c0 - plane) : nullptr);
    const float2* qzp2 = reinterpret_cast<const float2*>(p0f ? in.p0f + (k + 1 == nzu ? c0 - (nzu - 1) * plane : c0 + plane) : nullptr);
    const float2* qym2 = reinterpret_cast<const float2*>(p0f ? in.p0f + (has_ym ? c0 - nx : c0) : nullptr);
    const float2* qyp2 = reinterpret_cast<const float2*>(p0f ? in.p0f + (has_yp ? c0 + nx : c0) : nullptr);
    auto res = [&](df pc, df pxm, df pxp, df pym, df pyp, df pzm, df pzp, df fv) {
      const df p2 = df_ldexp2(pc);
      const df lx = df_subz(df_addz(pxp, pxm), p2);
      const df lz = df_subz(df_addz(pzp, pzm), p2);
      const df ly = df_subz(df_addz(pyp, pym), p2);
      const df lap = df_addz(df_addz(df_mulz(lx, lcx), df_mulz(ly, lcy)), df_mulz(lz, lcz));
      return df_to_f(df_subz(df_subz(fv, fmean), lap));
    };
    // the cells 2e, 2e+1 of the line with their neighbours, as pairs (P32: from
    // the FP32 p, low parts zero)
    auto cell2 = [&](int e, auto P32) -> cpx<T> {
      constexpr bool F = decltype(P32)::value;
      const int i0 = 2 * e;
      float4 c, zm, zp, ym, yp;
      df pxm, pxp;
      if constexpr (F) {
        const float2 c2 = qc2[e], zm2 = qzm2[e], zp2 = qzp2[e];
        c = make_float4(c2.x, 0.0f, c2.y, 0.0f);
        zm = make_float4(zm2.x, 0.0f, zm2.y, 0.0f);
        zp = make_float4(zp2.x, 0.0f, zp2.y, 0.0f);
        pxm = {ql[i0 == 0 ? nx - 1 : i0 - 1], 0.0f};
        pxp = {ql[i0 + 2 == nx ? 0 : i0 + 2], 0.0f};
        if (has_ym) {
          const float2 v = qym2[e];
          ym = make_float4(v.x, 0.0f, v.y, 0.0f);
        } else {
          ym = c;
        }
        if (has_yp) {
          const float2 v = qyp2[e];
          yp = make_float4(v.x, 0.0f, v.y, 0.0f);
        } else {
          yp = OPEN ? make_float4(-c.x, -c.y, -c.z, -c.w) : c;
        }
      } else {
        c = pc4[e];
        pxm = pl[i0 == 0 ? nx - 1 : i0 - 1];
        pxp = pl[i0 + 2 == nx ? 0 : i0 + 2];
        zm = pzm4[e];
        zp = pzp4[e];
        ym = has_ym ? pym4[e] : c;  // wall mirror below the bottom cell
        // above the top cell: the wall mirror, or the outflow ghost -p (p = 0 on the face)
        yp = has_yp ? pyp4[e] : (OPEN ? make_float4(-c.x, -c.y, -c.z, -c.w) : c);
      }
      const float4 fv = f4[e];
      const df a0 = {c.x, c.y}, a1 = {c.z, c.w};
      const float r0 = res(a0, pxm, a1, df{ym.x, ym.y}, df{yp.x, yp.y}, df{zm.x, zm.y}, df{zp.x, zp.y},
                           df{fv.x, fv.y});
      const float r1 = res(a1, a0, pxp, df{ym.z, ym.w}, df{yp.z, yp.w}, df{zm.z, zm.w}, df{zp.z, zp.w},
                           df{fv.z, fv.w});
      vmax = fmaxf(vmax, fmaxf(fabsf(r0), fabsf(r1)));
      return {r0, r1};
    };
    if (p0f)
      rgfft::run<T, false, M, 2, false>(
          [&](int e) -> cpx<T> { return valid ? cell2(e, std::true_type{}) : cpx<T>{(T)0, (T)0}; }, put,
          buf + ll * LS, 1, t0, tws);
    else
      rgfft::run<T, false, M, 2, false>(
          [&](int e) -> cpx<T> { return valid ? cell2(e, std::false_type{}) : cpx<T>{(T)0, (T)0}; }, put,
          buf + ll * LS, 1, t0, tws);
  }
  if (SRC == SRC_F) block_max_to(&sc->fmax_bits, vmax);
  else if (SRC == SRC_RESID) block_max_to(&sc->rmax_bits[slot], vmax);  // float max, widened once per warp
  if (SRC == SRC_F || SRC == SRC_FDF) {
    // per-CTA sum of f, totalled in a fixed order by the next kernel (finish_sums)
    block_pair_sums(fsum, df{0.0f, 0.0f}, sc->part + (size_t)g.ny * g.nz + bid);
    if (bid == 0 && threadIdx.x == 0) sc->x_parts = (int)nblk;
  }
  __syncthreads();
  // untangle: X_k = (Z_k + conj Z_{M-k})/2 - i W^k (Z_k - conj Z_{M-k})/2, W = exp(-2 pi i/nx)
  auto untangle = [&](int lq, int kx) {
    const cpx<T> zk = buf[lq * LS + rgfft::row(kx == M ? 0 : kx)];
    const cpx<T> zc = buf[lq * LS + rgfft::row(kx == 0 ? 0 : M - kx)];
    const cpx<T> a = {zk.x + zc.x, zk.y - zc.y};
    const cpx<T> b = {zk.x - zc.x, zk.y + zc.y};
    const cpx<T> wb = cmul(tws[kx], b);
    cpx<T> X;
    X.x = (T)0.5 * (a.x + wb.y);
    X.y = (T)0.5 * (a.y - wb.x);
    return X;
  };
  if constexpr (!PL) {
    for (int idx = threadIdx.x; idx < L * nxh; idx += blockDim.x) {
      const int lq = idx / nxh, kx = idx - lq * nxh;
      if (l0 + lq >= nlines) continue;
      spec[(l0 + lq) * (uint32_t)nxh + kx] = untangle(lq, kx);
    }
  } else {
    // transposed store: plane kx holds the lines in order (index kx * lines + line)
    const PlaneLanes pl = plane_lanes(L);
    const int lane = threadIdx.x & 31, lqo = lane % pl.lq, kxo = lane / pl.lq;
    const int ngl = L / pl.lq, ngk = (nxh + pl.kq - 1) / pl.kq;
    for (int w = threadIdx.x >> 5; w < ngl * ngk; w += blockDim.x >> 5) {
      const int gl = w % ngl, gk = w / ngl;
      const int lq = gl * pl.lq + lqo, kx = gk * pl.kq + kxo;
      if (kx >= nxh || l0 + lq >= nlines) continue;
      spec[(uint32_t)kx * nlines + l0 + lq] = untangle(lq, kx);
    }
  }
}
template <int SRC, int M, bool OPEN, bool PL = false>
__global__ void __launch_bounds__(256) k_xfwd_rg(GridDev g, StencilIn in, DevScalars* sc, int slot, df* fdf,
                                                 const df* __restrict__ pdf, cpx<float>* spec,
                                                 const cpx<float>* __restrict__ tw, int L) {
  pdl_enter();
  xfwd_rg_body<SRC, M, OPEN, PL>(g, in, sc, slot, fdf, pdf, spec, tw, L, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// z pass
// ---------------------------------------------------------------------------
template <typename T, bool INV, int N>
__device__ __forceinline__ void zfft_body(GridDev g, cpx<T>* spec, RadixPlan rp, const cpx<T>* tw,
                                              int tkx, const DevScalars* sc, DevScalars* fin, uint32_t bid, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (fin && bid == 0) finish_sums(fin, g);  // uniform over the CTA
  if (sc && sc->done) return;
  const int nz = g.nz, nxh = g.nx / 2 + 1;
  const int ntile = (nxh + tkx - 1) / tkx;
  const int j = bid / ntile;
  const int kx0 = (bid - j * ntile) * tkx;
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* b = a + (size_t)tkx * nz;
  cpx<T>* tws = b + (size_t)tkx * nz;  // exp(-2 pi i t/nz)
  for (int t = threadIdx.x; t < nz; t += blockDim.x) cp_async<sizeof(cpx<T>)>(&tws[t], &tw[t]);
  const size_t rowstride = (size_t)g.ny * nxh;
  const size_t base = (size_t)j * nxh + kx0;
  const int tl2 = ilog2_dev(tkx);
  for (int idx = threadIdx.x; idx < nz * tkx; idx += blockDim.x) {
    const int k = idx >> tl2, c = idx & (tkx - 1);
    if (kx0 + c < nxh)
      cp_async<sizeof(cpx<T>)>(&a[idx], &spec[base + k * rowstride + c]);
    else
      a[idx] = {(T)0, (T)0};
  }
  cp_async_wait_all();
  __syncthreads();
  cpx<T>* r = fft_any<T, INV, N, 1>(a, b, tl2, rp, 1, tkx, tws);
  for (int idx = threadIdx.x; idx < nz * tkx; idx += blockDim.x) {
    const int k = idx >> tl2, c = idx & (tkx - 1);
    if (kx0 + c < nxh) spec[base + k * rowstride + c] = r[idx];
  }
}
template <typename T, bool INV, int N>
__global__ void __launch_bounds__(256) k_zfft(GridDev g, cpx<T>* spec, RadixPlan rp, const cpx<T>* __restrict__ tw,
                                              int tkx, const DevScalars* sc, DevScalars* fin) {
  zfft_body<T, INV, N>(g, spec, rp, tw, tkx, sc, fin, blockIdx.x, gridDim.x);
}

// Register-staged z pass (FP32, power-of-two nz; rgfft in fft.cuh): one CTA
// per (j, tile of L kx columns), L * nz/16 threads; the first pass reads the
// columns from the spectrum and the last pass writes them back, so each
// element crosses shared memory once.
template <typename T, bool INV, int N>
__device__ __forceinline__ void zfft_rg_body(GridDev g, cpx<T>* spec, const cpx<T>* tw, int L,
                                                 const DevScalars* sc, DevScalars* fin, uint32_t bid, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (fin && bid == 0) finish_sums(fin, g);  // uniform over the CTA
  if (sc && sc->done) return;
  const uint32_t nxh = (uint32_t)g.nx / 2 + 1;
  const uint32_t ntile = (nxh + L - 1) / L;
  const uint32_t j = bid / ntile;
  const uint32_t kx0 = (bid - j * ntile) * L;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* tws = buf + rgfft::rows(N) * L;  // exp(-2 pi i t/nz)
  for (int t = threadIdx.x; t < N; t += blockDim.x) tws[t] = tw[t];
  const int line = threadIdx.x & (L - 1), t0 = threadIdx.x >> ilog2_dev(L);
  const bool valid = kx0 + line < nxh;
  const uint32_t rs = (uint32_t)g.ny * nxh;  // kz stride (32-bit offsets: spectra below 2^32 elements)
  cpx<T>* col = spec + (j * nxh + kx0 + line);
  rgfft::run<T, INV, N, 1, false>(
      [&](int e) { return valid ? col[(uint32_t)e * rs] : cpx<T>{(T)0, (T)0}; },
      [&](int e, cpx<T> v) {
        if (valid) col[(uint32_t)e * rs] = v;
      },
      buf + line, L, t0, tws);
}
template <typename T, bool INV, int N>
__global__ void __launch_bounds__(256) k_zfft_rg(GridDev g, cpx<T>* spec, const cpx<T>* __restrict__ tw, int L,
                                                 const DevScalars* sc, DevScalars* fin) {
  pdl_enter();
  zfft_rg_body<T, INV, N>(g, spec, tw, L, sc, fin, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// y pass: Neumann tridiagonal solve per (kx, kz)
// ---------------------------------------------------------------------------
// Row j of the system for one wavenumber pair, with a = 1/dy^2 and
// lam = lam_x(kx) + lam_z(kz):
//   row 0:       (-a + lam) x_0 + a x_1                 = d_0
//   0 < j < N-1: a x_{j-1} + (-2a + lam) x_j + a x_{j+1} = d_j
//   row N-1:     a x_{N-2} + (-a + lam) x_{N-1}         = d_{N-1}
// Thomas elimination with multipliers m_j = 1/(b_j - a * a m_{j-1}):
//   forward  x~_j = (d_j - a x~_{j-1}) m_j,  backward x_j = x~_j - a m_j x_{j+1}.
// The table holds, per line, [m_inf, m_{N-1}, m_0 .. m_{J-1}]: m_j equals m_inf
// bit for bit for J <= j <= N-2.  For kx = kz = 0 the matrix is singular (the
// constant mode): m_0 = 0 pins x_0 = 0, the mean of d is removed first and the
// mean of x afterwards, which gives the zero-mean solution.
// One thread per (kx, kz) line, walking the line in global memory: in the
// spectrum layout [kz][j][kx] the threads of a warp (consecutive kx) read and
// write 32 consecutive elements per j, and each sweep moves in chunks of 8
// elements whose loads (and multipliers) are issued before the chunk's
// recurrence runs.  Nothing is staged in shared memory, so every line of the
// spectrum has its thread resident at once (the shared-memory tile allowed
// about 16 lines per CTA).  Same arithmetic, in the same order, as the
// recurrences above.
template <typename T>
__global__ void __launch_bounds__(128) k_ythomas(GridDev g, cpx<T>* spec, const T* __restrict__ tab,
                                                 const int* __restrict__ line_off, const int* __restrict__ line_len,
                                                 T a, const DevScalars* sc) {
  if (sc && sc->done) return;
  const int nxh = g.nx / 2 + 1, ny = g.ny;
  const int kz = blockIdx.y;
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  if (kx >= nxh) return;  // no barriers below
  const int line = kz * nxh + kx;
  const int off = line_off[line], J = line_len[line];
  const T m_inf = tab[off], m_last = tab[off + 1];
  const size_t stride = (size_t)nxh;
  cpx<T>* col = spec + (size_t)kz * ny * nxh + kx;
  auto mult = [&](int jj) { return jj < J ? tab[off + 2 + jj] : (jj < ny - 1 ? m_inf : m_last); };
  const bool zero_line = !g.top_open && kz == 0 && kx == 0;  // the wall problem's singular line
  cpx<T> shift = {(T)0, (T)0};
  if (zero_line) {
    double sx = 0.0, sy = 0.0;
    for (int jj = 0; jj < ny; ++jj) {
      sx += (double)col[jj * stride].x;
      sy += (double)col[jj * stride].y;
    }
    shift.x = (T)(sx / ny);
    shift.y = (T)(sy / ny);
  }
  constexpr int C = 8;
  cpx<T> prev = {(T)0, (T)0};
  for (int j0 = 0; j0 < ny; j0 += C) {  // the last chunk may be short (ny = 2^a 3^b)
    cpx<T> d[C];
    T m[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      if (j0 + u < ny) {
        d[u] = col[(j0 + u) * stride];
        m[u] = mult(j0 + u);
      }
    }
#pragma unroll
    for (int u = 0; u < C; ++u) {
      if (j0 + u >= ny) break;
      cpx<T> v = d[u];
      v.x = (v.x - shift.x - a * prev.x) * m[u];
      v.y = (v.y - shift.y - a * prev.y) * m[u];
      col[(j0 + u) * stride] = v;
      prev = v;
    }
  }
  // backward: j = ny-2 .. 0 in chunks of 8 from the top
  for (int j1 = ny - 2; j1 >= 0; j1 -= C) {
    cpx<T> d[C];
    T m[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      const int jj = j1 - u;
      if (jj >= 0) {
        d[u] = col[jj * stride];
        m[u] = mult(jj);
      }
    }
#pragma unroll
    for (int u = 0; u < C; ++u) {
      const int jj = j1 - u;
      if (jj < 0) break;
      const T cj = a * m[u];
      cpx<T> v = d[u];
      v.x -= cj * prev.x;
      v.y -= cj * prev.y;
      col[jj * stride] = v;
      prev = v;
    }
  }
  if (zero_line) {
    double sx = 0.0, sy = 0.0;
    for (int jj = 0; jj < ny; ++jj) {
      sx += (double)col[jj * stride].x;
      sy += (double)col[jj * stride].y;
    }
    const T mx = (T)(sx / ny), my = (T)(sy / ny);
    for (int jj = 0; jj < ny; ++jj) {
      col[jj * stride].x -= mx;
      col[jj * stride].y -= my;
    }
  }
}

// y pass of the FP32 solve: DCT-II along y, divide by the eigenvalues of L,
// DCT-III back -- the cosine basis diagonalises the Neumann operator, so this
// equals the tridiagonal solve of k_ythomas but is fully parallel.  The
// DCT-II of a complex line x is formed from one FFT of the reordered line
// v[pos(j)] = x_j (pos(j) = j/2 for even j, N-1-(j-1)/2 for odd j; Makhoul
// 1980): X_k = (w_k V_k + conj(w_k) V_{N-k})/2 with w_k = exp(-i pi k/(2N)),
// V_N = V_0.  The inverse takes V'_k = conj(w_k)(P_k - i P_{N-k}), P_N = 0,
// an inverse FFT, and x_j = v'[pos(j)] / N.  Eigenvalue of mode (kx, ky, kz):
// lam_x[kx] + lam_y[ky] + lam_z[kz]; the zero mode is set to zero.
template <typename T, int N>
__device__ __forceinline__ void ydct_body(GridDev g, cpx<T>* spec, RadixPlan rp, const cpx<T>* tw,
                                              const cpx<T>* wq, const T* lam_x,
                                              const T* lam_y, const T* lam_z, int tky,
                                              const DevScalars* zsc, uint32_t bid, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nxh = g.nx / 2 + 1, ny = g.ny;
  const int ntile = (nxh + tky - 1) / tky;
  const int kz = bid / ntile, kx0 = (bid - kz * ntile) * tky;
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* b = a + (size_t)tky * ny;
  cpx<T>* tws = b + (size_t)tky * ny;  // exp(-2 pi i t/ny)
  for (int t = threadIdx.x; t < ny; t += blockDim.x) cp_async<sizeof(cpx<T>)>(&tws[t], &tw[t]);
  const int t2 = ilog2_dev(tky);
  const size_t base = (size_t)kz * ny * nxh + kx0;
  for (int idx = threadIdx.x; idx < ny * tky; idx += blockDim.x) {
    const int j = idx >> t2, c = idx & (tky - 1);
    const int pj = (j & 1) ? ny - 1 - (j >> 1) : (j >> 1);
    if (kx0 + c < nxh)
      cp_async<sizeof(cpx<T>)>(&a[pj * tky + c], &spec[base + (size_t)j * nxh + c]);
    else
      a[pj * tky + c] = {(T)0, (T)0};
  }
  cp_async_wait_all();
  __syncthreads();
  cpx<T>* V = fft_any<T, false, N, 1>(a, b, t2, rp, 1, tky, tws);
  const T inv_n = (T)1 / (T)ny;
  const T lz = lam_z[kz];
  const int npair = ny / 2 + 1;
  for (int idx = threadIdx.x; idx < npair * tky; idx += blockDim.x) {
    const int k = idx >> t2, c = idx & (tky - 1);
    const int kx = kx0 + c;
    if (kx >= nxh) continue;
    const T lxz = lam_x[kx] + lz;
    if (k == 0) {
      const T lam = lxz + lam_y[0];
      const cpx<T> v0 = V[c];
      if (kx == 0 && kz == 0) {  // zero mode pinned (to the value that keeps p zero-mean)
        V[c] = {(T)zsc->zmode, (T)0};
        continue;
      }
      const T s = inv_n / lam;
      V[c] = {v0.x * s, v0.y * s};
      continue;
    }
    const int r = ny - k;
    const cpx<T> vk = V[k * tky + c], vr = V[r * tky + c];
    const cpx<T> wk = wq[k], wr = wq[r];
    const cpx<T> wkc = {wk.x, -wk.y}, wrc = {wr.x, -wr.y};
    cpx<T> xk, xr;
    if constexpr (std::is_same<T, dd>::value) {
      // pairs: X_k = (w_k V_k + conj(w_k) V_r)/2 and X_r = (w_r V_r + conj(w_r) V_k)/2
      // share the sums V_k + V_r and the differences, so that each component
      // is half of one two-term dot product (w = a + i b):
      // Re X_k = (a (Re V_k + Re V_r) + b (Im V_r - Im V_k))/2, and likewise
      const dd s1 = dd_add_lazy(vk.x, vr.x), s2 = dd_add_lazy(vk.y, vr.y);
      const dd d1 = dd_sub_lazy(vr.y, vk.y), d2 = dd_sub_lazy(vk.x, vr.x);
      auto half = [](dd v) { return dd(0.5f * v.hi, 0.5f * v.lo); };
      xk = {half(dd_dot2<false>(wk.x, s1, wk.y, d1)), half(dd_dot2<false>(wk.x, s2, wk.y, d2))};
      xr = {half(dd_dot2<true>(wr.x, s1, wr.y, d1)), half(dd_dot2<true>(wr.x, s2, wr.y, d2))};
    } else {
      const cpx<T> t1 = cmul(wk, vk), t2c = cmul(wkc, vr);
      xk = {(T)0.5 * (t1.x + t2c.x), (T)0.5 * (t1.y + t2c.y)};
      const cpx<T> t3 = cmul(wr, vr), t4 = cmul(wrc, vk);
      xr = {(T)0.5 * (t3.x + t4.x), (T)0.5 * (t3.y + t4.y)};
    }
    const T sk = inv_n / (lxz + lam_y[k]), sr = inv_n / (lxz + lam_y[r]);
    const cpx<T> pk = {xk.x * sk, xk.y * sk}, pr = {xr.x * sr, xr.y * sr};
    // V'_k = conj(w_k)(P_k - i P_r), V'_r = conj(w_r)(P_r - i P_k);  -i z = (z.y, -z.x)
    V[k * tky + c] = cmul(wkc, cpx<T>{pk.x + pr.y, pk.y - pr.x});
    if (r != k) V[r * tky + c] = cmul(wrc, cpx<T>{pr.x + pk.y, pr.y - pk.x});
  }
  __syncthreads();
  cpx<T>* W = (V == a) ? b : a;
  cpx<T>* R = fft_any<T, true, N, 1>(V, W, t2, rp, 1, tky, tws);
  for (int idx = threadIdx.x; idx < ny * tky; idx += blockDim.x) {
    const int j = idx >> t2, c = idx & (tky - 1);
    const int pj = (j & 1) ? ny - 1 - (j >> 1) : (j >> 1);
    if (kx0 + c < nxh) spec[base + (size_t)j * nxh + c] = R[pj * tky + c];
  }
}
template <typename T, int N>
__global__ void __launch_bounds__(256) k_ydct(GridDev g, cpx<T>* spec, RadixPlan rp, const cpx<T>* __restrict__ tw,
                                              const cpx<T>* __restrict__ wq, const T* __restrict__ lam_x,
                                              const T* __restrict__ lam_y, const T* __restrict__ lam_z, int tky,
                                              const DevScalars* zsc) {
  ydct_body<T, N>(g, spec, rp, tw, wq, lam_x, lam_y, lam_z, tky, zsc, blockIdx.x, gridDim.x);
}

// Register-staged form of k_ydct (FP32, power-of-two ny; rgfft in fft.cuh):
// the reordered line is read straight from the spectrum by the first pass of
// the DCT-II's FFT, the eigenvalue division works on the shared buffer, and
// the last pass of the inverse writes the reordered result back.  Same
// arithmetic as k_ydct.
template <typename T, int N>
__device__ __forceinline__ void ydct_rg_body(GridDev g, cpx<T>* spec, const cpx<T>* tw,
                                                 const cpx<T>* wq, const T* lam_x,
                                                 const T* lam_y, const T* lam_z, int L,
                                                 const DevScalars* zsc, uint32_t bid, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t nxh = (uint32_t)g.nx / 2 + 1;
  const uint32_t ntile = (nxh + L - 1) / L;
  const uint32_t kz = bid / ntile, kx0 = (bid - kz * ntile) * L;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* tws = buf + rgfft::rows(N) * L;  // exp(-2 pi i t/ny)
  for (int t = threadIdx.x; t < N; t += blockDim.x) tws[t] = tw[t];
  const int lg = ilog2_dev(L);
  const int line = threadIdx.x & (L - 1), t0 = threadIdx.x >> lg;
  const bool valid = kx0 + line < nxh;
  cpx<T>* col = spec + (kz * (uint32_t)N * nxh + kx0 + line);
  // v[p] = x_j with p = j/2 (even j) or N-1-(j-1)/2 (odd j)
  auto jof = [](int p) { return p < N / 2 ? 2 * p : 2 * (N - 1 - p) + 1; };
  rgfft::run<T, false, N, 1, false>(
      [&](int p) { return valid ? col[(uint32_t)jof(p) * nxh] : cpx<T>{(T)0, (T)0}; },
      [&](int e, cpx<T> v) { buf[rgfft::row(e) * L + line] = v; }, buf + line, L, t0, tws);
  __syncthreads();
  const T inv_n = (T)1 / (T)N;
  const T lz = lam_z[kz];
  constexpr int npair = N / 2 + 1;
#pragma unroll 1
  for (int idx = threadIdx.x; idx < npair * L; idx += blockDim.x) {
    const int k = idx >> lg, c = idx & (L - 1);
    const uint32_t kx = kx0 + c;
    if (kx >= nxh) continue;
    const T lxz = lam_x[kx] + lz;
    cpx<T>* Vk = buf + rgfft::row(k) * L + c;
    if (k == 0) {
      const T lam = lxz + lam_y[0];
      const cpx<T> v0 = *Vk;
      // inv_n / lam as inv_n * (1/lam): inv_n is a power of two, so the correctly
      // rounded reciprocal times it is the correctly rounded quotient
      if (kx == 0 && kz == 0) {  // zero mode pinned (to the value that keeps p zero-mean)
        *Vk = {(T)zsc->zmode, (T)0};
        continue;
      }
      const T s = inv_n * rcp_of(lam);
      *Vk = {v0.x * s, v0.y * s};
      continue;
    }
    const int r = N - k;
    cpx<T>* Vr = buf + rgfft::row(r) * L + c;
    const cpx<T> vk = *Vk, vr = *Vr;
    const cpx<T> wk = wq[k], wr = wq[r];
    const cpx<T> wkc = {wk.x, -wk.y}, wrc = {wr.x, -wr.y};
    const cpx<T> t1 = cmul(wk, vk), t2c = cmul(wkc, vr);
    const cpx<T> xk = {(T)0.5 * (t1.x + t2c.x), (T)0.5 * (t1.y + t2c.y)};
    const cpx<T> t3 = cmul(wr, vr), t4 = cmul(wrc, vk);
    const cpx<T> xr = {(T)0.5 * (t3.x + t4.x), (T)0.5 * (t3.y + t4.y)};
    const T sk = inv_n * rcp_of(lxz + lam_y[k]), sr = inv_n * rcp_of(lxz + lam_y[r]);
    const cpx<T> pk = {xk.x * sk, xk.y * sk}, pr = {xr.x * sr, xr.y * sr};
    // V'_k = conj(w_k)(P_k - i P_r), V'_r = conj(w_r)(P_r - i P_k);  -i z = (z.y, -z.x)
    *Vk = cmul(wkc, cpx<T>{pk.x + pr.y, pk.y - pr.x});
    if (r != k) *Vr = cmul(wrc, cpx<T>{pr.x + pk.y, pr.y - pk.x});
  }
  __syncthreads();
  rgfft::run<T, true, N, 1, true>(
      [&](int e) { return buf[rgfft::row(e) * L + line]; },
      [&](int e, cpx<T> v) { buf[rgfft::row(e) * L + line] = v; }, buf + line, L, t0, tws);
  __syncthreads();
  // x_j = v'[p(j)]: copy-out row by row (j = idx / L), consecutive threads on consecutive columns
  for (int idx = threadIdx.x; idx < N * L; idx += blockDim.x) {
    const int jj = idx >> lg, c = idx & (L - 1);
    const int pj = (jj & 1) ? N - 1 - (jj >> 1) : (jj >> 1);
    if (kx0 + c < nxh) spec[kz * (uint32_t)N * nxh + (uint32_t)jj * nxh + kx0 + c] = buf[rgfft::row(pj) * L + c];
  }
}
template <typename T, int N>
__global__ void __launch_bounds__(256, 4) k_ydct_rg(GridDev g, cpx<T>* spec, const cpx<T>* __restrict__ tw,
                                                 const cpx<T>* __restrict__ wq, const T* __restrict__ lam_x,
                                                 const T* __restrict__ lam_y, const T* __restrict__ lam_z, int L,
                                                 const DevScalars* zsc) {
  pdl_enter();
  ydct_rg_body<T, N>(g, spec, tw, wq, lam_x, lam_y, lam_z, L, zsc, blockIdx.x, gridDim.x);
}

// 256-point form of k_ydct_rg (radices 16 x 16) with the eigenvalue divide in
// registers between the transforms.  After the second forward pass thread t
// holds X_k for k = t + 16 q, which is the set the first inverse pass reads,
// so only the partners X_{N-k} (held by thread 16 - t) cross shared memory.
// Each thread forms V'_k for its own k with the operations k_ydct_rg uses for
// that member of the pair (k, N-k) (the compiler may contract products into
// sums differently, so the last bits can differ; the FP32 solve is refined).
__device__ __forceinline__ void ydct256_body(GridDev g, cpx<float>* spec, const cpx<float>* tw,
                                                  const cpx<float>* wq, const float* lam_x,
                                                  const float* lam_y, const float* lam_z,
                                                  int L, const DevScalars* zsc, uint32_t bid, uint32_t nblk) {
  using T = float;
  constexpr int N = 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t nxh = (uint32_t)g.nx / 2 + 1;
  const uint32_t ntile = (nxh + L - 1) / L;
  const uint32_t kz = bid / ntile, kx0 = (bid - kz * ntile) * L;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* tws = buf + rgfft::rows(N) * L;  // exp(-2 pi i t/ny)
  for (int t = threadIdx.x; t < N; t += blockDim.x) tws[t] = tw[t];
  const int lg = ilog2_dev(L);
  const int line = threadIdx.x & (L - 1), t0 = threadIdx.x >> lg;  // t0 in [0, 16)
  const uint32_t kx = kx0 + line;
  const bool valid = kx < nxh;
  cpx<T>* col = spec + (kz * (uint32_t)N * nxh + kx);
  cpx<T>* ln = buf + line;
  // v[p] = x_j with p = j/2 (even j) or N-1-(j-1)/2 (odd j)
  auto jof = [](int p) { return p < N / 2 ? 2 * p : 2 * (N - 1 - p) + 1; };
  cpx<T> v[16];
  // forward pass 0 (the DCT-II's reordered line straight from the spectrum)
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = valid ? col[(uint32_t)jof(t0 + 16 * q) * nxh] : cpx<T>{(T)0, (T)0};
  SmallDft<T, false, 16>::run(v);
#pragma unroll
  for (int q = 0; q < 16; ++q) ln[rgfft::row(16 * t0 + q) * L] = v[q];
  __syncthreads();
  // forward pass 1: v[q] = X_{t0 + 16 q}
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = ln[rgfft::row(t0 + 16 * q) * L];
#pragma unroll
  for (int q = 1; q < 16; ++q) v[q] = cmul(v[q], tws[q * t0]);
  SmallDft<T, false, 16>::run(v);
  __syncthreads();  // every read of pass 1 before the exchange writes
#pragma unroll
  for (int q = 0; q < 16; ++q) ln[rgfft::row(t0 + 16 * q) * L] = v[q];
  __syncthreads();
  // divide by the eigenvalues (zero mode pinned); V'_k = conj(w_k)(P_k - i P_r)
  const T inv_n = (T)1 / (T)N;
  const T lxz = (valid ? lam_x[kx] : (T)0) + lam_z[kz];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int k = t0 + 16 * q;
    if (k == 0) {
      // inv_n / lam as inv_n * (1/lam): inv_n is a power of two
      if (kx == 0 && kz == 0) {  // zero mode pinned (to the value that keeps p zero-mean)
        v[0] = {(T)zsc->zmode, (T)0};
        continue;
      }
      const T s0 = inv_n * __frcp_rn(lxz + lam_y[0]);
      v[0] = {v[0].x * s0, v[0].y * s0};
      continue;
    }
    const int r = N - k;
    const cpx<T> vk = v[q], vr = ln[rgfft::row(r) * L];
    const cpx<T> wk = wq[k], wr = wq[r];
    const cpx<T> wkc = {wk.x, -wk.y}, wrc = {wr.x, -wr.y};
    const cpx<T> t1 = cmul(wk, vk), t2c = cmul(wkc, vr);
    const cpx<T> xk = {(T)0.5 * (t1.x + t2c.x), (T)0.5 * (t1.y + t2c.y)};
    const cpx<T> t3 = cmul(wr, vr), t4 = cmul(wrc, vk);
    const cpx<T> xr = {(T)0.5 * (t3.x + t4.x), (T)0.5 * (t3.y + t4.y)};
    const T sk = inv_n * __frcp_rn(lxz + lam_y[k]), sr = inv_n * __frcp_rn(lxz + lam_y[r]);
    const cpx<T> pk = {xk.x * sk, xk.y * sk}, pr = {xr.x * sr, xr.y * sr};
    v[q] = cmul(wkc, cpx<T>{pk.x + pr.y, pk.y - pr.x});
  }
  __syncthreads();  // the partners' reads before the inverse overwrites the buffer
  // inverse pass 0 from registers
  SmallDft<T, true, 16>::run(v);
#pragma unroll
  for (int q = 0; q < 16; ++q) ln[rgfft::row(16 * t0 + q) * L] = v[q];
  __syncthreads();
  // inverse pass 1: outputs t0 + 16 q, back to the spectrum in physical order
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = ln[rgfft::row(t0 + 16 * q) * L];
#pragma unroll
  for (int q = 1; q < 16; ++q) {
    cpx<T> w = tws[q * t0];
    w.y = -w.y;
    v[q] = cmul(v[q], w);
  }
  SmallDft<T, true, 16>::run(v);
  if (valid) {
#pragma unroll
    for (int q = 0; q < 16; ++q) col[(uint32_t)jof(t0 + 16 * q) * nxh] = v[q];
  }
}
static __global__ void __launch_bounds__(256, 4) k_ydct256(GridDev g, cpx<float>* spec, const cpx<float>* __restrict__ tw,
                                                  const cpx<float>* __restrict__ wq, const float* __restrict__ lam_x,
                                                  const float* __restrict__ lam_y, const float* __restrict__ lam_z,
                                                  int L, const DevScalars* zsc) {
  pdl_enter();
  ydct256_body(g, spec, tw, wq, lam_x, lam_y, lam_z, L, zsc, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// inverse x pass
// ---------------------------------------------------------------------------
// MODE: XI_F64 p = s x (FP64); XI_DF pdf = s x (pairs); XI_DF_ACC pdf += s x
template <typename T, int MODE, int N>
__device__ __forceinline__ void xinv_body(GridDev g, const cpx<T>* spec, double* p, df* pdf,
                                              double scale, RadixPlan rp, const cpx<T>* tw, int lpb,
                                              const DevScalars* sc, DevScalars* psc, uint32_t bid, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (sc && sc->done) return;
  const int nx = g.nx, M = nx / 2, nxh = M + 1;
  const int lsc = M + 1;  // line stride (complex): nxh values, also the padded FFT stride
  const int nlines = g.ny * g.nz;
  const int l0 = bid * lpb;
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smem_raw);  // lpb * lsc
  cpx<T>* b = a + (size_t)lpb * lsc;                // lpb * lsc
  cpx<T>* tws = b + (size_t)lpb * lsc;              // exp(-2 pi i t/nx), t < nx
  for (int t = threadIdx.x; t < nx; t += blockDim.x) cp_async<sizeof(cpx<T>)>(&tws[t], &tw[t]);
  for (int idx = threadIdx.x; idx < lpb * nxh; idx += blockDim.x) {
    const int ll = (int)fdiv(idx, g.fd_nxh);
    const int line = l0 + ll;
    if (line < nlines)
      cp_async<sizeof(cpx<T>)>(&b[idx], &spec[(size_t)l0 * nxh + idx]);
    else
      b[idx] = {(T)0, (T)0};
  }
  cp_async_wait_all();
  __syncthreads();
  // Z_k = E_k + i O_k, E = (X_k + conj X_{M-k})/2, O = (X_k - conj X_{M-k}) conj(W^k)/2
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int ll = (int)fdiv(idx, g.fd_m), k = idx - ll * M;
    const cpx<T> xk = b[ll * lsc + k];
    const cpx<T> xc = b[ll * lsc + (M - k)];
    const cpx<T> e = {(T)0.5 * (xk.x + xc.x), (T)0.5 * (xk.y - xc.y)};
    cpx<T> dd = {(T)0.5 * (xk.x - xc.x), (T)0.5 * (xk.y + xc.y)};
    cpx<T> w = tws[k];
    w.y = -w.y;
    const cpx<T> o = cmul(dd, w);
    a[ll * lsc + k] = {e.x - o.y, e.y + o.x};
  }
  __syncthreads();
  cpx<T>* z = fft_any<T, true, N, 2>(a, b, ilog2_dev(lpb), rp, lsc, 1, tws);
  const df sdf = d2df(scale);
  df psum = {0.0f, 0.0f};  // sum of the p written (pairs)
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int ll = (int)fdiv(idx, g.fd_m), n = idx - ll * M;
    const int line = l0 + ll;
    if (line >= nlines) continue;
    const cpx<T> v = z[ll * lsc + n];
    const size_t o = (size_t)line * nx + 2 * n;
    if constexpr (std::is_same<T, dd>::value) {
      // pairs: scaled in pair arithmetic, written as FP64 or pairs
      const df d0 = df_mul(sdf, v.x.pair()), d1 = df_mul(sdf, v.y.pair());
      if (MODE == XI_F64) {
        p[o] = df2d(d0);
        p[o + 1] = df2d(d1);
      } else if (MODE == XI_DF) {
        reinterpret_cast<float4*>(pdf)[o >> 1] = make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
        psum = df_addz(df_addz(psum, d0), d1);
      } else {
        const float4 q = reinterpret_cast<const float4*>(pdf)[o >> 1];
        const df s0 = df_add(df{q.x, q.y}, d0), s1 = df_add(df{q.z, q.w}, d1);
        reinterpret_cast<float4*>(pdf)[o >> 1] = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
        psum = df_addz(df_addz(psum, s0), s1);
      }
    } else if (MODE == XI_F64) {
      p[o] = scale * (double)v.x;
      p[o + 1] = scale * (double)v.y;
    } else {
      const df d0 = df_mul_f(sdf, (float)v.x), d1 = df_mul_f(sdf, (float)v.y);
      if (MODE == XI_DF) {
        reinterpret_cast<float4*>(pdf)[o >> 1] = make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
        psum = df_addz(df_addz(psum, d0), d1);
      } else {
        const float4 q = reinterpret_cast<const float4*>(pdf)[o >> 1];
        const df s0 = df_add(df{q.x, q.y}, d0), s1 = df_add(df{q.z, q.w}, d1);
        reinterpret_cast<float4*>(pdf)[o >> 1] = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
        psum = df_addz(df_addz(psum, s0), s1);
      }
    }
  }
  if (MODE != XI_F64 && psc) {
    // per-CTA sum of p, totalled in a fixed order by the next z pass (finish_sums)
    block_pair_sums(psum, df{0.0f, 0.0f}, psc->part + 2 * (size_t)g.ny * g.nz + bid);
    if (bid == 0 && threadIdx.x == 0) psc->p_parts = (int)nblk;
  }
}
template <typename T, int MODE, int N>
__global__ void __launch_bounds__(256) k_xinv(GridDev g, const cpx<T>* __restrict__ spec, double* p, df* pdf,
                                              double scale, RadixPlan rp, const cpx<T>* __restrict__ tw, int lpb,
                                              const DevScalars* sc, DevScalars* psc) {
  xinv_body<T, MODE, N>(g, spec, p, pdf, scale, rp, tw, lpb, sc, psc, blockIdx.x, gridDim.x);
}

// Register-staged inverse x pass (FP32, nx = 2M, M a power of two): thread
// (line, t) forms the packed values Z_k of its first inverse-FFT pass from
// X_k and X_{M-k} read straight from the spectrum, and the last pass stores
// (or adds) the real pairs of cells 2n, 2n+1 with one 16-byte access.  Same
// arithmetic as k_xinv.
// PL: the spectrum in the plane layout [kx][line]; the CTA's half spectra are
// first copied (transposed) into the shared buffer, then the first pass reads
// them there.
template <int MODE, int M, bool PL = false>
__device__ __forceinline__ void xinv_rg_body(GridDev g, const cpx<float>* spec, double* p, df* pdf,
                                                 double scale, const cpx<float>* tw, int L,
                                                 const DevScalars* sc, DevScalars* psc, uint32_t bid, uint32_t nblk,
                                                 float* p32 = nullptr) {
  using T = float;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (sc && sc->done) return;
  constexpr int TPL = M / 16, nx = 2 * M, nxh = M + 1, LS = xstride<PL>(M);
  const uint32_t nlines = (uint32_t)g.ny * (uint32_t)g.nz;
  const int ll = (int)threadIdx.x / TPL, t0 = (int)threadIdx.x & (TPL - 1);
  const uint32_t line = bid * (uint32_t)L + ll;
  const bool valid = line < nlines;
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* tws = buf + L * LS;
  for (int t = threadIdx.x; t < nx; t += blockDim.x) tws[t] = tw[t];
  if constexpr (PL) {
    const uint32_t l0 = bid * (uint32_t)L;
    const PlaneLanes pl = plane_lanes(L);
    const int lane = threadIdx.x & 31, lqo = lane % pl.lq, kxo = lane / pl.lq;
    const int ngl = L / pl.lq, ngk = (nxh + pl.kq - 1) / pl.kq;
    const int nw = (int)blockDim.x >> 5;
    // eight loads per thread in flight before their shared-memory stores
    constexpr int U = 8;
    for (int w0 = threadIdx.x >> 5; w0 < ngl * ngk; w0 += U * nw) {
      cpx<T> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int w = w0 + u * nw;
        const int gl = w % ngl, gk = w / ngl;
        const int lq = gl * pl.lq + lqo, kx = gk * pl.kq + kxo;
        v[u] = (w < ngl * ngk && kx < nxh && l0 + lq < nlines) ? spec[(uint32_t)kx * nlines + l0 + lq]
                                                                : cpx<T>{(T)0, (T)0};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int w = w0 + u * nw;
        const int gl = w % ngl, gk = w / ngl;
        const int lq = gl * pl.lq + lqo, kx = gk * pl.kq + kxo;
        if (w < ngl * ngk && kx < nxh) buf[lq * LS + rgfft::row(kx)] = v[u];
      }
    }
    __syncthreads();
  }
  const cpx<T>* X = PL ? nullptr : spec + line * (uint32_t)nxh;
  const cpx<T>* Xs = buf + ll * LS;
  const uint32_t c0 = line * (uint32_t)nx;
  const df sdf = d2df(scale);
  df psum = {0.0f, 0.0f};  // sum of the p written (pairs)
  // Z_k = E_k + i O_k, E = (X_k + conj X_{M-k})/2, O = (X_k - conj X_{M-k}) conj(W^k)/2
  auto ld = [&](int k) -> cpx<T> {
    if (!valid) return {(T)0, (T)0};
    const cpx<T> xk = PL ? Xs[rgfft::row(k)] : X[k];
    const cpx<T> xc = PL ? Xs[rgfft::row(M - k)] : X[M - k];
    const cpx<T> e = {(T)0.5 * (xk.x + xc.x), (T)0.5 * (xk.y - xc.y)};
    const cpx<T> dd = {(T)0.5 * (xk.x - xc.x), (T)0.5 * (xk.y + xc.y)};
    cpx<T> w = tw[k];
    w.y = -w.y;
    const cpx<T> o = cmul(dd, w);
    return {e.x - o.y, e.y + o.x};
  };
  auto st = [&](int n, cpx<T> v) {
    if (!valid) return;
    const uint32_t o = c0 + 2 * (uint32_t)n;
    if (MODE == XI_F64) {
      reinterpret_cast<double2*>(p)[o >> 1] = make_double2(scale * (double)v.x, scale * (double)v.y);
    } else if (MODE == XI_F32) {
      // the pair s x has a zero low part (s a power of two): its high part is p
      const df d0 = df_mul_f(sdf, (float)v.x), d1 = df_mul_f(sdf, (float)v.y);
      reinterpret_cast<float2*>(p32)[o >> 1] = make_float2(d0.hi, d1.hi);
      psum = df_addz(df_addz(psum, d0), d1);
    } else {
      const df d0 = df_mul_f(sdf, (float)v.x), d1 = df_mul_f(sdf, (float)v.y);
      float4* q4 = reinterpret_cast<float4*>(pdf) + (o >> 1);
      if (MODE == XI_DF) {
        *q4 = make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
        psum = df_addz(df_addz(psum, d0), d1);
      } else {
        const float4 q = *q4;
        const df s0 = df_add(df{q.x, q.y}, d0), s1 = df_add(df{q.z, q.w}, d1);
        *q4 = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
      }
    }
  };
  if constexpr (MODE != XI_DF_ACC) {
    rgfft::run<T, true, M, 2, PL, rgfft::PAD_ROWS>(ld, st, buf + ll * LS, 1, t0, tws);
  } else {
    // p += s x: the last pass leaves x in shared memory; the update then runs
    // over consecutive cell pairs with four read-modify-writes in flight
    rgfft::run<T, true, M, 2, PL, rgfft::PAD_ROWS>(ld, [&](int e, cpx<T> v) { buf[ll * LS + rgfft::row(e)] = v; },
                                  buf + ll * LS, 1, t0, tws);
    __syncthreads();
    const uint32_t l0 = bid * (uint32_t)L;
    // the first sweep adds to the first solve's p in FP32 where it was kept so
    // (a pair with a zero low part: the same sums)
    const bool from32 = p32 != nullptr && psc != nullptr && psc->iter == 1;
    // U cell pairs in flight per thread: their old p (four floats as pairs, two
    // as FP32 -- twice as many loads for the same registers), then the updates
    auto update = [&](auto UC, auto F32) {
      constexpr int U = decltype(UC)::value;
      constexpr bool FROM32 = decltype(F32)::value;
      using Old = typename std::conditional<FROM32, float2, float4>::type;
      for (int b0 = threadIdx.x; b0 < L * M; b0 += U * blockDim.x) {
        Old q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = b0 + u * blockDim.x;
          const int lq = idx / M;
          if (idx < L * M && l0 + lq < nlines)
            q[u] = reinterpret_cast<const Old*>(FROM32 ? (const void*)p32 : (const void*)pdf)
                [(l0 + lq) * (uint32_t)M + (idx - lq * M)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = b0 + u * blockDim.x;
          const int lq = idx / M, n = idx - lq * M;
          if (idx >= L * M || l0 + lq >= nlines) continue;
          const cpx<T> v = buf[lq * LS + rgfft::row(n)];
          const df d0 = df_mul_f(sdf, (float)v.x), d1 = df_mul_f(sdf, (float)v.y);
          df a0, a1;
          if constexpr (FROM32) {
            a0 = {q[u].x, 0.0f};
            a1 = {q[u].y, 0.0f};
          } else {
            a0 = {q[u].x, q[u].y};
            a1 = {q[u].z, q[u].w};
          }
          const df s0 = df_add(a0, d0), s1 = df_add(a1, d1);
          reinterpret_cast<float4*>(pdf)[(l0 + lq) * (uint32_t)M + n] = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
          psum = df_addz(df_addz(psum, s0), s1);
        }
      }
    };
    if (from32)
      update(std::integral_constant<int, 8>{}, std::true_type{});
    else
      update(std::integral_constant<int, 4>{}, std::false_type{});
  }
  if (MODE != XI_F64 && psc) {
    // per-CTA sum of p, totalled in a fixed order by the next z pass (finish_sums)
    block_pair_sums(psum, df{0.0f, 0.0f}, psc->part + 2 * (size_t)g.ny * g.nz + bid);
    if (bid == 0 && threadIdx.x == 0) psc->p_parts = (int)nblk;
  }
}
template <int MODE, int M, bool PL = false>
__global__ void __launch_bounds__(256) k_xinv_rg(GridDev g, const cpx<float>* __restrict__ spec, double* p, df* pdf,
                                                 double scale, const cpx<float>* __restrict__ tw, int L,
                                                 const DevScalars* sc, DevScalars* psc, float* p32) {
  pdl_enter();
  xinv_rg_body<MODE, M, PL>(g, spec, p, pdf, scale, tw, L, sc, psc, blockIdx.x, gridDim.x, p32);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Lines per CTA of the register-staged passes: the tuned tile, raised so that a
// CTA (L * N/16 threads) holds at least one full warp and capped so that it
// holds at most 256 threads (the kernels' launch bound).
// (nx/2) nz a power of two: the inverse transforms' scaling 1/((nx/2) nz) is exact in FP32
inline bool is_pow2_scale(const GridDev& g) {
  const unsigned m = (unsigned)(g.nx / 2) * (unsigned)g.nz;
  return m != 0u && (m & (m - 1u)) == 0u;
}

template <int N>
int rg_lines(int tile) {
  constexpr int lo = 32 / (N / 16) > 1 ? 32 / (N / 16) : 1, hi = 256 / (N / 16);
  return tile < lo ? lo : (tile > hi ? hi : tile);
}
template <typename T>
size_t rg_smem(int n, int L) {
  return sizeof(cpx<T>) * ((size_t)rgfft::rows(n) * L + (size_t)n);
}
// Lines per CTA of the register-staged x passes: the tuned x_lines, kept
// within one warp .. 256 threads (M/16 threads per line).
template <int M>
int rg_xlines(int lpb) {
  const int lo = 32 / (M / 16) > 1 ? 32 / (M / 16) : 1, hi = 256 / (M / 16);
  return lpb < lo ? lo : (lpb > hi ? hi : lpb);
}
inline size_t xrg_smem(int nx, int L, bool pl = false) {
  return sizeof(cpx<float>) * ((size_t)(pl ? xrg_stride_pl(nx / 2) : xrg_stride(nx / 2)) * L + (size_t)nx);
}

template <typename T>
size_t xfwd_smem(int nx, int lpb) {
  return sizeof(cpx<T>) * (2 * (size_t)lpb * (nx / 2 + 1) + (size_t)nx);
}
template <typename T>
size_t zfft_smem(int nz, int tkx) {
  return sizeof(cpx<T>) * (2 * (size_t)tkx * nz + (size_t)nz);
}
template <typename T>
size_t xinv_smem(int nx, int lpb) {
  return sizeof(cpx<T>) * (2 * (size_t)lpb * (nx / 2 + 1) + (size_t)nx);
}

template <typename T>
size_t xpass_smem_limit() {
  // every x-pass instance carries the same static reduction scratch (block_pair_sums)
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, k_xfwd<T, SRC_F, true, 0>) != cudaSuccess) return 0;
  return kSmemPerCta - a.sharedSizeBytes;
}

template <typename T>
size_t zpass_smem_limit() {
  // the z pass carries the static scratch of finish_sums
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, k_zfft<T, false, 0>) != cudaSuccess) return 0;
  return kSmemPerCta - a.sharedSizeBytes;
}

template <typename T>
cudaError_t set_smem_limits() {
  return set_rhs_smem_limit();
}

template <typename T>
cudaError_t launch_xfwd(int src, bool do_fft, const GridDev& g, const StencilIn& in, DevScalars* sc, int slot,
                        df* fdf, const df* pdf, cpx<T>* spec, const RadixPlan& rp, const cpx<T>* tw, int lpb,
                        cudaStream_t st) {
  const int nlines = g.ny * g.nz;
  const int grid = (nlines + lpb - 1) / lpb;
  const size_t sm = xfwd_smem<T>(g.nx, lpb);
  return with_len<T>(g.nx / 2, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    cudaError_t e;
    if constexpr (sizeof(T) == 4 && rgfft::is_rg<N>::value) {
      // (the register-staged form reads f with 16-byte loads)
      // (the plane layout has only these instances: f must be 16-byte aligned)
      if (do_fft && (src != SRC_F || ((uintptr_t)in.f & 15u) == 0 || g.spec_planes)) {
        const int L = rg_xlines<N>(lpb);
        const int gr = (nlines + L - 1) / L;
        const size_t smr = xrg_smem(g.nx, L, g.spec_planes != 0);
        auto go = [&](auto kernel) -> cudaError_t {
          cudaError_t e2 = allow_smem(kernel, smr);
          if (e2 != cudaSuccess) return e2;
          launch_pdl(kernel, gr, L * (N / 16), smr, st, g, in, sc, slot, fdf, pdf, (cpx<float>*)spec, (const cpx<float>*)tw, L);
          return cudaGetLastError();
        };
        if (g.spec_planes) {
          if (src == SRC_F) return go(k_xfwd_rg<SRC_F, N, false, true>);
          if (src == SRC_FDF) return go(k_xfwd_rg<SRC_FDF, N, false, true>);
          return go(k_xfwd_rg<SRC_RESID, N, false, true>);  // the plane layout has walls only
        }
        if (src == SRC_F) return go(k_xfwd_rg<SRC_F, N, false>);
        if (src == SRC_FDF) return go(k_xfwd_rg<SRC_FDF, N, false>);
        if (!g.top_open) return go(k_xfwd_rg<SRC_RESID, N, false>);
        return go(k_xfwd_rg<SRC_RESID, N, true>);
      }
    }
    if (g.spec_planes) return cudaErrorInvalidValue;  // plane layout: power-of-two nx/2 only
    if (src == SRC_F) {
      if ((e = allow_smem(k_xfwd<T, SRC_F, true, N>, sm)) != cudaSuccess) return e;
      k_xfwd<T, SRC_F, true, N><<<grid, 256, sm, st>>>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb);
    } else if (src == SRC_FDF) {
      if ((e = allow_smem(k_xfwd<T, SRC_FDF, true, N>, sm)) != cudaSuccess) return e;
      k_xfwd<T, SRC_FDF, true, N><<<grid, 256, sm, st>>>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb);
    } else if (do_fft && !g.top_open) {
      if ((e = allow_smem(k_xfwd<T, SRC_RESID, true, N>, sm)) != cudaSuccess) return e;
      k_xfwd<T, SRC_RESID, true, N><<<grid, 256, sm, st>>>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb);
    } else if (do_fft) {
      if ((e = allow_smem(k_xfwd<T, SRC_RESID, true, N, true>, sm)) != cudaSuccess) return e;
      k_xfwd<T, SRC_RESID, true, N, true><<<grid, 256, sm, st>>>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb);
    } else if (!g.top_open) {
      if ((e = allow_smem(k_xfwd<T, SRC_RESID, false, 0>, sm)) != cudaSuccess) return e;
      k_xfwd<T, SRC_RESID, false, 0><<<grid, 256, sm, st>>>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb);
    } else {
      if ((e = allow_smem(k_xfwd<T, SRC_RESID, false, 0, true>, sm)) != cudaSuccess) return e;
      k_xfwd<T, SRC_RESID, false, 0, true><<<grid, 256, sm, st>>>(g, in, sc, slot, fdf, pdf, spec, rp, tw, lpb);
    }
    return cudaGetLastError();
  });
}


template <typename T>
cudaError_t launch_zfft(bool inverse, const GridDev& g, cpx<T>* spec, const RadixPlan& rp, const cpx<T>* tw,
                        int tkx, const DevScalars* sc, DevScalars* fin, cudaStream_t st) {
  const int nxh = g.nx / 2 + 1;
  const int grid = g.ny * ((nxh + tkx - 1) / tkx);
  const size_t sm = zfft_smem<T>(g.nz, tkx);
  return with_len<T>(g.nz, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    cudaError_t e;
    if constexpr (has_ct_lengths<T>::value && rgfft::is_rg<N>::value) {
      const int L = rg_lines<N>(tkx);
      const int gr = g.ny * ((nxh + L - 1) / L);
      const size_t smr = rg_smem<T>(N, L);
      if (inverse) {
        if ((e = allow_smem(k_zfft_rg<T, true, N>, smr)) != cudaSuccess) return e;
        launch_pdl(k_zfft_rg<T, true, N>, gr, L * (N / 16), smr, st, g, spec, tw, L, sc, fin);
      } else {
        if ((e = allow_smem(k_zfft_rg<T, false, N>, smr)) != cudaSuccess) return e;
        launch_pdl(k_zfft_rg<T, false, N>, gr, L * (N / 16), smr, st, g, spec, tw, L, sc, fin);
      }
      return cudaGetLastError();
    }
    if (inverse) {
      if ((e = allow_smem(k_zfft<T, true, N>, sm)) != cudaSuccess) return e;
      k_zfft<T, true, N><<<grid, 256, sm, st>>>(g, spec, rp, tw, tkx, sc, fin);
    } else {
      if ((e = allow_smem(k_zfft<T, false, N>, sm)) != cudaSuccess) return e;
      k_zfft<T, false, N><<<grid, 256, sm, st>>>(g, spec, rp, tw, tkx, sc, fin);
    }
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_ythomas(const GridDev& g, cpx<T>* spec, const T* tab, const int* off, const int* len, T a,
                           const DevScalars* sc, cudaStream_t st) {
  const int nxh = g.nx / 2 + 1;
  const dim3 grid((nxh + 127) / 128, g.nz);
  k_ythomas<T><<<grid, 128, 0, st>>>(g, spec, tab, off, len, a, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ydct(const GridDev& g, cpx<T>* spec, const RadixPlan& rp, const cpx<T>* tw, const cpx<T>* wq,
                        const T* lam_x, const T* lam_y, const T* lam_z, int tky, const DevScalars* zsc,
                        cudaStream_t st) {
  const int nxh = g.nx / 2 + 1;
  const int grid = g.nz * ((nxh + tky - 1) / tky);
  const size_t sm = zfft_smem<T>(g.ny, tky);
  return with_len<T>(g.ny, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    // (FP32 only: the register-staged y pass in pairs needs ~190 registers, one
    // CTA per SM, and ran 1.6x slower than the shared-memory form at 256^3)
    if constexpr (sizeof(T) == 4 && rgfft::is_rg<N>::value) {
      const int L = rg_lines<N>(tky);
      const int gr = g.nz * ((nxh + L - 1) / L);
      const size_t smr = rg_smem<T>(N, L);
      if constexpr (N == 256 && sizeof(T) == 4) {
        cudaError_t e = allow_smem(k_ydct256, smr);
        if (e != cudaSuccess) return e;
        launch_pdl(k_ydct256, gr, L * (N / 16), smr, st, g, (cpx<float>*)spec, (const cpx<float>*)tw,
                                                 (const cpx<float>*)wq, (const float*)lam_x, (const float*)lam_y,
                                                 (const float*)lam_z, L, zsc);
        return cudaGetLastError();
      }
      cudaError_t e = allow_smem(k_ydct_rg<T, N>, smr);
      if (e != cudaSuccess) return e;
      launch_pdl(k_ydct_rg<T, N>, gr, L * (N / 16), smr, st, g, spec, tw, wq, lam_x, lam_y, lam_z, L, zsc);
      return cudaGetLastError();
    }
    cudaError_t e = allow_smem(k_ydct<T, N>, sm);
    if (e != cudaSuccess) return e;
    k_ydct<T, N><<<grid, 256, sm, st>>>(g, spec, rp, tw, wq, lam_x, lam_y, lam_z, tky, zsc);
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_xinv(int mode, const GridDev& g, const cpx<T>* spec, double* p, df* pdf, double scale,
                        const RadixPlan& rp, const cpx<T>* tw, int lpb, const DevScalars* sc, DevScalars* psc,
                        cudaStream_t st, float* p32) {
  const int nlines = g.ny * g.nz;
  const int grid = (nlines + lpb - 1) / lpb;
  const size_t sm = xinv_smem<T>(g.nx, lpb);
  return with_len<T>(g.nx / 2, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    cudaError_t e;
    // (the register-staged form writes an FP64 p with 16-byte stores)
    if constexpr (sizeof(T) == 4 && rgfft::is_rg<N>::value) {
      if (mode != XI_F64 || ((uintptr_t)p & 15u) == 0 || g.spec_planes) {
      if (mode == XI_F64 && ((uintptr_t)p & 15u) != 0) return cudaErrorMisalignedAddress;
      const int L = rg_xlines<N>(lpb);
      const int gr = (nlines + L - 1) / L;
      const size_t smr = xrg_smem(g.nx, L, g.spec_planes != 0);
      auto go = [&](auto kernel) -> cudaError_t {
        cudaError_t e2 = allow_smem(kernel, smr);
        if (e2 != cudaSuccess) return e2;
        launch_pdl(kernel, gr, L * (N / 16), smr, st, g, (const cpx<float>*)spec, p, pdf, scale, (const cpx<float>*)tw, L,
                                               sc, psc, p32);
        return cudaGetLastError();
      };
      if (mode == XI_F32 && !(p32 && is_pow2_scale(g))) return cudaErrorInvalidValue;
      if (g.spec_planes) {
        if (mode == XI_F64) return go(k_xinv_rg<XI_F64, N, true>);
        if (mode == XI_DF) return go(k_xinv_rg<XI_DF, N, true>);
        if (mode == XI_F32) return go(k_xinv_rg<XI_F32, N, true>);
        return go(k_xinv_rg<XI_DF_ACC, N, true>);
      }
      if (mode == XI_F64) return go(k_xinv_rg<XI_F64, N>);
      if (mode == XI_DF) return go(k_xinv_rg<XI_DF, N>);
      if (mode == XI_F32) return go(k_xinv_rg<XI_F32, N>);
      return go(k_xinv_rg<XI_DF_ACC, N>);
      }
    }
    if (mode == XI_F32 || p32) return cudaErrorInvalidValue;  // FP32 p: the register-staged passes only
    if (g.spec_planes) return cudaErrorInvalidValue;  // plane layout: power-of-two nx/2 only
    if (mode == XI_F64) {
      if ((e = allow_smem(k_xinv<T, XI_F64, N>, sm)) != cudaSuccess) return e;
      k_xinv<T, XI_F64, N><<<grid, 256, sm, st>>>(g, spec, p, pdf, scale, rp, tw, lpb, sc, psc);
    } else if (mode == XI_DF) {
      if ((e = allow_smem(k_xinv<T, XI_DF, N>, sm)) != cudaSuccess) return e;
      k_xinv<T, XI_DF, N><<<grid, 256, sm, st>>>(g, spec, p, pdf, scale, rp, tw, lpb, sc, psc);
    } else {
      if ((e = allow_smem(k_xinv<T, XI_DF_ACC, N>, sm)) != cudaSuccess) return e;
      k_xinv<T, XI_DF_ACC, N><<<grid, 256, sm, st>>>(g, spec, p, pdf, scale, rp, tw, lpb, sc, psc);
    }
    return cudaGetLastError();
  });
}

#define PPE_INST(T)                                                                                              \
  template size_t xfwd_smem<T>(int, int);                                                                        \
  template size_t zfft_smem<T>(int, int);                                                                        \
  template size_t xinv_smem<T>(int, int);                                                                        \
  template cudaError_t set_smem_limits<T>();                                                                     \
  template size_t xpass_smem_limit<T>();                                                                         \
  template cudaError_t launch_xfwd<T>(int, bool, const GridDev&, const StencilIn&, DevScalars*, int, df*,       \
                                      const df*, cpx<T>*, const RadixPlan&, const cpx<T>*, int, cudaStream_t);  \
  template cudaError_t launch_zfft<T>(bool, const GridDev&, cpx<T>*, const RadixPlan&, const cpx<T>*, int,      \
                                      const DevScalars*, DevScalars*, cudaStream_t);                             \
  template size_t zpass_smem_limit<T>();                                                                         \
  template cudaError_t launch_ythomas<T>(const GridDev&, cpx<T>*, const T*, const int*, const int*, T,          \
                                         const DevScalars*, cudaStream_t);                                       \
  template cudaError_t launch_ydct<T>(const GridDev&, cpx<T>*, const RadixPlan&, const cpx<T>*, const cpx<T>*,     \
                                      const T*, const T*, const T*, int, const DevScalars*, cudaStream_t);       \
  template cudaError_t launch_xinv<T>(int, const GridDev&, const cpx<T>*, double*, df*, double,                  \
                                      const RadixPlan&, const cpx<T>*, int, const DevScalars*, DevScalars*,      \
                                      cudaStream_t, float*);


}  // namespace ppe
