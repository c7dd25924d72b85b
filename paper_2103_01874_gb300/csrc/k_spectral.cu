// Spectral kernels of the direct Poisson solve of Eq. (34) (the fast Poisson
// solver stated after Eq. (34): periodic x and z, homogeneous Neumann walls in y).
//
// Spectrum layout (plan workspace): complex T, [kz][j][kx] with kx fastest,
// kx = 0 .. nx/2 (nxh = nx/2 + 1 values, the real-input half spectrum), j the
// physical wall-normal index, kz = 0 .. nz-1.  Every pass works in place.
//
//   k_xfwd    one CTA per `lpb` x-lines: builds the real line (Eq. (34) RHS,
//             a given f, or the residual f - L p), packs it as nx/2 complex
//             values, FFTs them and untangles the nx/2+1 half spectrum.
//   k_zfft    one CTA per (j, tile of `tkx` kx columns): FFT along z.
//   k_ythomas one thread per (kx, kz): the Neumann tridiagonal solve in y with
//             precomputed elimination multipliers; zero mode pinned.
//   k_xinv    one CTA per `lpb` lines: half spectrum -> real line, scaled, and
//             stored to p or added to p (refinement update).
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

template <typename T>
__device__ __forceinline__ cpx<T> ld_tw(const cpx<T>* tw, int t) {
  return tw[t];
}

// ---------------------------------------------------------------------------
// forward x pass
// ---------------------------------------------------------------------------
template <typename T, int SRC, bool DO_FFT>
__global__ void __launch_bounds__(256) k_xfwd(GridDev g, StencilIn in, DevScalars* sc, int slot, double* f_out,
                                              cpx<T>* spec, RadixPlan rp, const cpx<T>* __restrict__ tw, int lpb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (SRC == SRC_RESID && sc->done) return;
  const int nx = g.nx, M = nx / 2, nxh = M + 1;
  const int nlines = g.ny * g.nz;
  const int l0 = blockIdx.x * lpb;
  T* line_re = reinterpret_cast<T*>(smem_raw);                       // lpb * nx reals == lpb * M complex
  cpx<T>* bufb = reinterpret_cast<cpx<T>*>(smem_raw + sizeof(T) * (size_t)lpb * nx);

  double rho0 = 0.0;
  if (SRC == SRC_RHS) rho0 = read_rho0(sc);
  double vmax = 0.0;
  for (int idx = threadIdx.x; idx < lpb * nx; idx += blockDim.x) {
    const int ll = idx / nx, i = idx - ll * nx;
    const int line = l0 + ll;
    double val = 0.0;
    if (line < nlines) {
      const int k = line / g.ny, j = line - k * g.ny;
      if (SRC == SRC_RHS) {
        val = rhs_at(g, in, rho0, i, j, k);
        if (f_out) f_out[(size_t)line * nx + i] = val;
      } else if (SRC == SRC_F) {
        val = __ldg(in.f + (size_t)line * nx + i);
      } else {
        val = resid_at(g, in, i, j, k);
      }
      vmax = fmax(vmax, fabs(val));
    }
    line_re[idx] = (T)val;
  }
  if (SRC == SRC_RHS || SRC == SRC_F) block_max_to(&sc->fmax_bits, vmax);
  else block_max_to(&sc->rmax_bits[slot], vmax);
  if (!DO_FFT) return;
  __syncthreads();
  cpx<T>* z = fft_lines<T, false>(reinterpret_cast<cpx<T>*>(line_re), bufb, lpb, rp, M, 1, tw, 2, false);
  // untangle: X_k = (Z_k + conj Z_{M-k})/2 - i W^k (Z_k - conj Z_{M-k})/2, W = exp(-2 pi i/nx)
  for (int idx = threadIdx.x; idx < lpb * nxh; idx += blockDim.x) {
    const int ll = idx / nxh, kx = idx - ll * nxh;
    const int line = l0 + ll;
    if (line >= nlines) continue;
    const cpx<T> zk = z[ll * M + (kx == M ? 0 : kx)];
    const cpx<T> zc = z[ll * M + (kx == 0 ? 0 : M - kx)];
    const cpx<T> a = {zk.x + zc.x, zk.y - zc.y};
    const cpx<T> b = {zk.x - zc.x, zk.y + zc.y};
    const cpx<T> wb = cmul(ld_tw(tw, kx), b);
    cpx<T> X;
    X.x = (T)0.5 * (a.x + wb.y);
    X.y = (T)0.5 * (a.y - wb.x);
    spec[(size_t)line * nxh + kx] = X;
  }
}

// ---------------------------------------------------------------------------
// z pass
// ---------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_zfft(GridDev g, cpx<T>* spec, RadixPlan rp, const cpx<T>* __restrict__ tw,
                                              int tkx, const DevScalars* sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (sc && sc->done) return;
  const int nz = g.nz, nxh = g.nx / 2 + 1;
  const int ntile = (nxh + tkx - 1) / tkx;
  const int j = blockIdx.x / ntile;
  const int kx0 = (blockIdx.x - j * ntile) * tkx;
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* b = a + (size_t)tkx * nz;
  const size_t rowstride = (size_t)g.ny * nxh;
  const size_t base = (size_t)j * nxh + kx0;
  for (int idx = threadIdx.x; idx < nz * tkx; idx += blockDim.x) {
    const int k = idx / tkx, c = idx - k * tkx;
    cpx<T> v = {(T)0, (T)0};
    if (kx0 + c < nxh) v = spec[base + k * rowstride + c];
    a[idx] = v;
  }
  __syncthreads();
  cpx<T>* r = fft_lines<T, INV>(a, b, tkx, rp, 1, tkx, tw, 1, true);
  for (int idx = threadIdx.x; idx < nz * tkx; idx += blockDim.x) {
    const int k = idx / tkx, c = idx - k * tkx;
    if (kx0 + c < nxh) spec[base + k * rowstride + c] = r[idx];
  }
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
template <typename T>
__global__ void __launch_bounds__(128) k_ythomas(GridDev g, cpx<T>* spec, const T* __restrict__ tab,
                                                 const int* __restrict__ line_off, const int* __restrict__ line_len,
                                                 T a, const DevScalars* sc) {
  if (sc && sc->done) return;
  const int nxh = g.nx / 2 + 1, ny = g.ny;
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= nxh * g.nz) return;
  const int kx = line % nxh, kz = line / nxh;
  cpx<T>* d = spec + (size_t)kz * ny * nxh + kx;
  const size_t st = nxh;
  const int off = line_off[line], J = line_len[line];
  const T m_inf = tab[off], m_last = tab[off + 1];
  const T* mj = tab + off + 2;
  cpx<T> shift = {(T)0, (T)0};
  if (line == 0) {
    double sx = 0.0, sy = 0.0;
    for (int j = 0; j < ny; ++j) {
      sx += (double)d[j * st].x;
      sy += (double)d[j * st].y;
    }
    shift.x = (T)(sx / ny);
    shift.y = (T)(sy / ny);
  }
  cpx<T> prev = {(T)0, (T)0};
  for (int j = 0; j < ny; ++j) {
    const T m = (j < J) ? mj[j] : ((j < ny - 1) ? m_inf : m_last);
    cpx<T> v = d[j * st];
    v.x = (v.x - shift.x - a * prev.x) * m;
    v.y = (v.y - shift.y - a * prev.y) * m;
    d[j * st] = v;
    prev = v;
  }
  for (int j = ny - 2; j >= 0; --j) {
    const T m = (j < J) ? mj[j] : m_inf;
    const T c = a * m;
    cpx<T> v = d[j * st];
    v.x -= c * prev.x;
    v.y -= c * prev.y;
    d[j * st] = v;
    prev = v;
  }
  if (line == 0) {
    double sx = 0.0, sy = 0.0;
    for (int j = 0; j < ny; ++j) {
      sx += (double)d[j * st].x;
      sy += (double)d[j * st].y;
    }
    const T mx = (T)(sx / ny), my = (T)(sy / ny);
    for (int j = 0; j < ny; ++j) {
      cpx<T> v = d[j * st];
      v.x -= mx;
      v.y -= my;
      d[j * st] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// inverse x pass
// ---------------------------------------------------------------------------
template <typename T, bool ACCUM>
__global__ void __launch_bounds__(256) k_xinv(GridDev g, const cpx<T>* __restrict__ spec, double* p, double scale,
                                              RadixPlan rp, const cpx<T>* __restrict__ tw, int lpb,
                                              const DevScalars* sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (sc && sc->done) return;
  const int nx = g.nx, M = nx / 2, nxh = M + 1;
  const int nlines = g.ny * g.nz;
  const int l0 = blockIdx.x * lpb;
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smem_raw);  // lpb * M
  cpx<T>* b = a + (size_t)lpb * M;                  // lpb * (M + 1)
  for (int idx = threadIdx.x; idx < lpb * nxh; idx += blockDim.x) {
    const int ll = idx / nxh;
    const int line = l0 + ll;
    cpx<T> v = {(T)0, (T)0};
    if (line < nlines) v = spec[(size_t)l0 * nxh + idx];
    b[idx] = v;
  }
  __syncthreads();
  // Z_k = E_k + i O_k, E = (X_k + conj X_{M-k})/2, O = (X_k - conj X_{M-k}) conj(W^k)/2
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int ll = idx / M, k = idx - ll * M;
    const cpx<T> xk = b[ll * nxh + k];
    const cpx<T> xc = b[ll * nxh + (M - k)];
    const cpx<T> e = {(T)0.5 * (xk.x + xc.x), (T)0.5 * (xk.y - xc.y)};
    cpx<T> dd = {(T)0.5 * (xk.x - xc.x), (T)0.5 * (xk.y + xc.y)};
    cpx<T> w = ld_tw(tw, k);
    w.y = -w.y;
    const cpx<T> o = cmul(dd, w);
    a[idx] = {e.x - o.y, e.y + o.x};
  }
  __syncthreads();
  cpx<T>* z = fft_lines<T, true>(a, b, lpb, rp, M, 1, tw, 2, false);
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int ll = idx / M, n = idx - ll * M;
    const int line = l0 + ll;
    if (line >= nlines) continue;
    const cpx<T> v = z[idx];
    double* out = p + (size_t)line * nx + 2 * n;
    const double v0 = scale * (double)v.x, v1 = scale * (double)v.y;
    if (ACCUM) {
      out[0] += v0;
      out[1] += v1;
    } else {
      out[0] = v0;
      out[1] = v1;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
size_t xfwd_smem(int nx, int lpb) {
  return sizeof(T) * (size_t)lpb * nx + sizeof(cpx<T>) * (size_t)lpb * (nx / 2);
}
template <typename T>
size_t zfft_smem(int nz, int tkx) {
  return 2 * sizeof(cpx<T>) * (size_t)tkx * nz;
}
template <typename T>
size_t xinv_smem(int nx, int lpb) {
  return sizeof(cpx<T>) * (size_t)lpb * (nx / 2) + sizeof(cpx<T>) * (size_t)lpb * (nx / 2 + 1);
}

template <typename T>
cudaError_t set_smem_limits() {
  const int lim = 227 * 1024;
  cudaError_t e = cudaSuccess;
#define PPE_SET(K) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
  PPE_SET((k_xfwd<T, SRC_RHS, true>));
  PPE_SET((k_xfwd<T, SRC_RHS, false>));
  PPE_SET((k_xfwd<T, SRC_F, true>));
  PPE_SET((k_xfwd<T, SRC_RESID, true>));
  PPE_SET((k_xfwd<T, SRC_RESID, false>));
  PPE_SET((k_zfft<T, false>));
  PPE_SET((k_zfft<T, true>));
  PPE_SET((k_xinv<T, false>));
  PPE_SET((k_xinv<T, true>));
#undef PPE_SET
  return e;
}

template <typename T>
cudaError_t launch_xfwd(int src, bool do_fft, const GridDev& g, const StencilIn& in, DevScalars* sc, int slot,
                        double* f_out, cpx<T>* spec, const RadixPlan& rp, const cpx<T>* tw, int lpb,
                        cudaStream_t st) {
  const int nlines = g.ny * g.nz;
  const int grid = (nlines + lpb - 1) / lpb;
  const size_t sm = do_fft ? xfwd_smem<T>(g.nx, lpb) : sizeof(T) * (size_t)lpb * g.nx;
  if (src == SRC_RHS && do_fft)
    k_xfwd<T, SRC_RHS, true><<<grid, 256, sm, st>>>(g, in, sc, slot, f_out, spec, rp, tw, lpb);
  else if (src == SRC_RHS)
    k_xfwd<T, SRC_RHS, false><<<grid, 256, sm, st>>>(g, in, sc, slot, f_out, spec, rp, tw, lpb);
  else if (src == SRC_F)
    k_xfwd<T, SRC_F, true><<<grid, 256, sm, st>>>(g, in, sc, slot, f_out, spec, rp, tw, lpb);
  else if (do_fft)
    k_xfwd<T, SRC_RESID, true><<<grid, 256, sm, st>>>(g, in, sc, slot, f_out, spec, rp, tw, lpb);
  else
    k_xfwd<T, SRC_RESID, false><<<grid, 256, sm, st>>>(g, in, sc, slot, f_out, spec, rp, tw, lpb);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zfft(bool inverse, const GridDev& g, cpx<T>* spec, const RadixPlan& rp, const cpx<T>* tw,
                        int tkx, const DevScalars* sc, cudaStream_t st) {
  const int nxh = g.nx / 2 + 1;
  const int grid = g.ny * ((nxh + tkx - 1) / tkx);
  const size_t sm = zfft_smem<T>(g.nz, tkx);
  if (inverse)
    k_zfft<T, true><<<grid, 256, sm, st>>>(g, spec, rp, tw, tkx, sc);
  else
    k_zfft<T, false><<<grid, 256, sm, st>>>(g, spec, rp, tw, tkx, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ythomas(const GridDev& g, cpx<T>* spec, const T* tab, const int* off, const int* len, T a,
                           const DevScalars* sc, cudaStream_t st) {
  const int lines = (g.nx / 2 + 1) * g.nz;
  k_ythomas<T><<<(lines + 127) / 128, 128, 0, st>>>(g, spec, tab, off, len, a, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xinv(bool accumulate, const GridDev& g, const cpx<T>* spec, double* p, double scale,
                        const RadixPlan& rp, const cpx<T>* tw, int lpb, const DevScalars* sc, cudaStream_t st) {
  const int nlines = g.ny * g.nz;
  const int grid = (nlines + lpb - 1) / lpb;
  const size_t sm = xinv_smem<T>(g.nx, lpb);
  if (accumulate)
    k_xinv<T, true><<<grid, 256, sm, st>>>(g, spec, p, scale, rp, tw, lpb, sc);
  else
    k_xinv<T, false><<<grid, 256, sm, st>>>(g, spec, p, scale, rp, tw, lpb, sc);
  return cudaGetLastError();
}

#define PPE_INST(T)                                                                                              \
  template size_t xfwd_smem<T>(int, int);                                                                        \
  template size_t zfft_smem<T>(int, int);                                                                        \
  template size_t xinv_smem<T>(int, int);                                                                        \
  template cudaError_t set_smem_limits<T>();                                                                     \
  template cudaError_t launch_xfwd<T>(int, bool, const GridDev&, const StencilIn&, DevScalars*, int, double*,    \
                                      cpx<T>*, const RadixPlan&, const cpx<T>*, int, cudaStream_t);             \
  template cudaError_t launch_zfft<T>(bool, const GridDev&, cpx<T>*, const RadixPlan&, const cpx<T>*, int,      \
                                      const DevScalars*, cudaStream_t);                                          \
  template cudaError_t launch_ythomas<T>(const GridDev&, cpx<T>*, const T*, const int*, const int*, T,          \
                                         const DevScalars*, cudaStream_t);                                       \
  template cudaError_t launch_xinv<T>(bool, const GridDev&, const cpx<T>*, double*, double, const RadixPlan&,   \
                                      const cpx<T>*, int, const DevScalars*, cudaStream_t);
PPE_INST(double)
PPE_INST(float)
#undef PPE_INST

}  // namespace ppe
