// Point-wise kernels of the projection: rho_0 = min(rho) (text after Eq. (32)),
// the velocity correction of Eq. (33), and the device-side refinement control.
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

// keep_rho0: leave rho_0 as the last right-hand side set it (ppe_solve).
__global__ void k_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0) {
  if (threadIdx.x != 0) return;
  // rho0 <= 0: start the min-reduction at +inf
  if (!keep_rho0)
    sc->rho0_bits = rho0 > 0.0 ? (unsigned long long)__double_as_longlong(rho0) : 0x7FF0000000000000ull;
  sc->last_slot = -1;
  sc->fmax_bits = 0ull;
  for (int s = 0; s < kMaxSweeps + 2; ++s) sc->rmax_bits[s] = 0ull;
  sc->done = 0;
  sc->sweeps = 0;
  sc->iter = 1;
  sc->cont = 0;
  sc->tol = tol;
}

__global__ void __launch_bounds__(256) k_rho_min(const double* __restrict__ rho, size_t n, DevScalars* sc) {
  double m = __longlong_as_double(0x7FF0000000000000ll);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmin(m, __ldg(rho + i));
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  // rho > 0, so the bit patterns order like the values
  if ((threadIdx.x & 31) == 0) atomicMin(&sc->rho0_bits, (unsigned long long)__double_as_longlong(m));
}

// Eq. (33) after the solve, from the explicitly split velocity u_pre written by
// the right-hand-side kernel:  u^{n+1} = u_pre - (dt/rho_0) G p^{n+1}.
// One thread per (i, j, k) with 0 <= j <= ny: x and z faces of cell (i, j, k)
// (j < ny) and the y face j; wall faces keep v_pre (= v*).  p is read as pairs
// (pdf) or as FP64 (p64); with both given, p64 receives p in FP64.
__global__ void __launch_bounds__(256) k_correct_pre(GridDev g, double dt, const df* __restrict__ upre,
                                                     const df* __restrict__ vpre, const df* __restrict__ wpre,
                                                     const df* __restrict__ pdf, double* p64, const DevScalars* sc,
                                                     double* u_out, double* v_out, double* w_out) {
  const size_t nx = (size_t)g.nx, ny = (size_t)g.ny;
  const size_t total = (size_t)g.nz * (ny + 1) * nx;
  const StencilConst K = sc->K;
  auto P = [&](size_t c) -> df { return pdf ? pdf[c] : d2df(p64[c]); };
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = fdiv((uint32_t)t, g.fd_nx);
    const int i = (int)((uint32_t)t - r * (uint32_t)nx);
    const int k = (int)fdiv(r, g.fd_nyp1);
    const int j = (int)(r - (uint32_t)k * (uint32_t)(ny + 1));
    const size_t cv = t;  // v index (k*(ny+1) + j)*nx + i
    if (j == 0 || j == g.ny) {
      v_out[cv] = df2d(vpre[cv]);
      if (j == g.ny) continue;
    }
    const Nbr n = neighbours(g, i, j, k);
    const df p0 = P(n.c);
    if (j > 0) v_out[cv] = df2d(df_sub(vpre[cv], df_mul(K.gy, df_sub(p0, P(n.c - nx)))));
    u_out[n.c] = df2d(df_sub(upre[n.c], df_mul(K.gx, df_sub(p0, P(n.xm)))));
    w_out[n.c] = df2d(df_sub(wpre[n.c], df_mul(K.gz, df_sub(p0, P(n.zm)))));
    if (pdf && p64) p64[n.c] = df2d(p0);
  }
}

// Eq. (33) from the raw inputs:  u^{n+1} = u* - (dt/rho_0)(G p - beta_f G p_hat),
// using 1/rho_f - 1/rho_0 = -beta_f/rho_0.  In-place (u_out == u) is allowed:
// every thread reads u*, v*, w* only at the faces it writes.
__global__ void __launch_bounds__(256) k_correct_full(GridDev g, StencilIn in, const DevScalars* sc, double* u_out,
                                                      double* v_out, double* w_out) {
  const size_t nx = (size_t)g.nx, ny = (size_t)g.ny;
  const size_t total = (size_t)g.nz * (ny + 1) * nx;
  const StencilConst K = sc->K;
  const int rule = in.face_rule;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = fdiv((uint32_t)t, g.fd_nx);
    const int i = (int)((uint32_t)t - r * (uint32_t)nx);
    const int k = (int)fdiv(r, g.fd_nyp1);
    const int j = (int)(r - (uint32_t)k * (uint32_t)(ny + 1));
    const size_t cv = t;
    if (j == 0 || j == g.ny) {
      v_out[cv] = in.v[cv];
      if (j == g.ny) continue;
    }
    const Nbr n = neighbours(g, i, j, k);
    const df p0 = d2df(in.p[n.c]), h0 = phat_df(in.pn, in.pnm1, n.c), r0 = d2df(__ldg(in.rho + n.c));
    auto face = [&](size_t cn, const df& gk) -> df {
      const df b = beta_df(d2df(__ldg(in.rho + cn)), r0, K, rule);
      const df gp = df_sub(p0, d2df(in.p[cn]));
      const df gh = df_sub(h0, phat_df(in.pn, in.pnm1, cn));
      return df_mul(gk, df_sub(gp, df_mul(b, gh)));
    };
    if (j > 0) v_out[cv] = df2d(df_sub(d2df(in.v[cv]), face(n.c - nx, K.gy)));
    u_out[n.c] = df2d(df_sub(d2df(in.u[n.c]), face(n.xm, K.gx)));
    w_out[n.c] = df2d(df_sub(d2df(in.w[n.c]), face(n.zm, K.gz)));
  }
}

__global__ void __launch_bounds__(256) k_df_to_d(const df* __restrict__ a, double* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = df2d(a[i]);
}

// Test of the residual r_s = f - L p after s-1 corrections (slot s = iter):
// converged if ||r_s||_inf <= tol ||f||_inf; otherwise ask for correction s if
// s <= smax, else stop unconverged.  `sweeps` counts applied corrections.
__global__ void k_refine_check(DevScalars* sc, int smax, cudaGraphConditionalHandle handle, int use_handle) {
  if (threadIdx.x != 0) return;
  const int s = sc->iter;
  const double r = __longlong_as_double((long long)sc->rmax_bits[s]);
  const double f = __longlong_as_double((long long)sc->fmax_bits);
  sc->last_slot = s;
  int cont = 0;
  if (r <= sc->tol * f) {
    sc->done = 1;
    sc->sweeps = s - 1;
  } else if (s <= smax) {
    sc->sweeps = s;
    sc->iter = s + 1;
    cont = 1;
  } else {
    sc->sweeps = smax;
  }
  sc->cont = cont;
  if (use_handle) cudaGraphSetConditional(handle, cont);
}

__global__ void k_make_const(GridDev g, DevScalars* sc, double dt) {
  if (threadIdx.x == 0) sc->K = make_const(g, read_rho0(sc), dt);
}

__global__ void k_set_rho0(DevScalars* sc, double rho0) {
  if (threadIdx.x == 0) sc->rho0_bits = (unsigned long long)__double_as_longlong(rho0);
}

namespace {
unsigned grid_for(size_t total, size_t cap) {
  size_t b = (total + 255) / 256;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (unsigned)b;
}
}  // namespace

cudaError_t launch_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, cudaStream_t st) {
  k_init_scalars<<<1, 32, 0, st>>>(sc, rho0, tol, keep_rho0);
  return cudaGetLastError();
}

cudaError_t launch_set_rho0(DevScalars* sc, double rho0, cudaStream_t st) {
  k_set_rho0<<<1, 32, 0, st>>>(sc, rho0);
  return cudaGetLastError();
}

cudaError_t launch_make_const(const GridDev& g, DevScalars* sc, double dt, cudaStream_t st) {
  k_make_const<<<1, 32, 0, st>>>(g, sc, dt);
  return cudaGetLastError();
}

cudaError_t launch_rho_min(const double* rho, size_t n, DevScalars* sc, cudaStream_t st) {
  k_rho_min<<<grid_for(n, 152 * 8), 256, 0, st>>>(rho, n, sc);
  return cudaGetLastError();
}

cudaError_t launch_correct_pre(const GridDev& g, double dt, const df* upre, const df* vpre, const df* wpre,
                               const df* pdf, double* p64, const DevScalars* sc, double* u_out, double* v_out,
                               double* w_out, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  k_correct_pre<<<grid_for(total, (size_t)152 * 64), 256, 0, st>>>(g, dt, upre, vpre, wpre, pdf, p64, sc, u_out,
                                                                   v_out, w_out);
  return cudaGetLastError();
}

cudaError_t launch_correct_full(const GridDev& g, const StencilIn& in, const DevScalars* sc, double* u_out,
                                double* v_out, double* w_out, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  k_correct_full<<<grid_for(total, (size_t)152 * 64), 256, 0, st>>>(g, in, sc, u_out, v_out, w_out);
  return cudaGetLastError();
}

cudaError_t launch_df_to_d(const df* a, double* out, size_t n, cudaStream_t st) {
  k_df_to_d<<<grid_for(n, (size_t)152 * 32), 256, 0, st>>>(a, out, n);
  return cudaGetLastError();
}

cudaError_t launch_refine_check(DevScalars* sc, int smax, cudaGraphConditionalHandle handle, int use_handle,
                                cudaStream_t st) {
  k_refine_check<<<1, 32, 0, st>>>(sc, smax, handle, use_handle);
  return cudaGetLastError();
}

}  // namespace ppe
