// Point-wise kernels of the projection: rho_0 = min(rho) (text after Eq. (32)),
// the velocity correction of Eq. (33), and the device-side refinement control.
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "pdl.cuh"
#include "stencil.cuh"
#include "correct.cuh"

namespace ppe {

__global__ void k_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, double* out_p,
                               double* out_u, double* out_v, double* out_w) {
  pdl_enter();
  if (threadIdx.x == 0) init_scalars(sc, rho0, tol, keep_rho0, out_p, out_u, out_v, out_w);
}

__global__ void __launch_bounds__(256) k_rho_min(const double* __restrict__ rho, size_t n, DevScalars* sc) {
  pdl_enter();
  rho_min_body(rho, n, sc, blockIdx.x, gridDim.x);
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
  const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
  const uint32_t total = (uint32_t)g.nz * (ny + 1) * nx;
  const StencilConst K = sc->K;
  auto P = [&](size_t c) -> df { return pdf ? pdf[c] : d2df(p64[c]); };
  constexpr int U = 2;  // faces per thread per round, loads issued first
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x; t0 < total; t0 += U * stride) {
    df vp[U], up[U], wp[U], p0[U], pym[U], pxm[U], pzm[U];
    size_t cc[U];
    int jj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t t = t0 + u * stride;
      jj[u] = -1;
      if (t >= total) continue;
      const uint32_t r = fdiv(t, g.fd_nx);
      const int i = (int)(t - r * nx);
      const int k = (int)fdiv(r, g.fd_nyp1);
      const int j = (int)(r - (uint32_t)k * (ny + 1));
      jj[u] = j;
      vp[u] = vpre[t];
      if (j < (int)ny) {
        const Nbr n = neighbours(g, i, j, k);
        cc[u] = n.c;
        up[u] = upre[n.c];
        wp[u] = wpre[n.c];
        p0[u] = P(n.c);
        pxm[u] = P(n.xm);
        pzm[u] = P(n.zm);
        pym[u] = (j > 0) ? P(n.c - nx) : p0[u];
      } else if (g.top_open) {
        p0[u] = P(((size_t)k * ny + (ny - 1)) * nx + i);  // the top cell below the open face
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = jj[u];
      if (j < 0) continue;
      const uint32_t t = t0 + u * stride;
      if (j == (int)ny && g.top_open) {  // open top: the ghost -p of the cell below
        v_out[t] = df2d(df_subz(vp[u], df_mulz(K.gy, df_subz(df_neg(p0[u]), p0[u]))));
        continue;
      }
      if (j == 0 || j == (int)ny) {
        v_out[t] = df2d(vp[u]);
        if (j == (int)ny) continue;
      } else {
        v_out[t] = df2d(df_subz(vp[u], df_mulz(K.gy, df_subz(p0[u], pym[u]))));
      }
      const size_t c = cc[u];
      u_out[c] = df2d(df_subz(up[u], df_mulz(K.gx, df_subz(p0[u], pxm[u]))));
      w_out[c] = df2d(df_subz(wp[u], df_mulz(K.gz, df_subz(p0[u], pzm[u]))));
      if (pdf && p64) p64[c] = df2d(p0[u]);
    }
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
    if (j == g.ny && g.top_open) {
      // open top: the face between the top cell and its ghost (-p, -p_hat, same density)
      const size_t ct = ((size_t)k * ny + (ny - 1)) * nx + i;
      const df pt = d2df(in.p[ct]), ht = phat_df(in.pn, in.pnm1, ct), rt = d2df(__ldg(in.rho + ct));
      const df b = beta_df(rt, rt, K, rule);
      const df gp = df_subz(df_neg(pt), pt), gh = df_subz(df_neg(ht), ht);
      v_out[cv] = df2d(df_subz(d2df(in.v[cv]), df_mulz(K.gy, df_subz(gp, df_mulz(b, gh)))));
      continue;
    }
    if (j == 0 || j == g.ny) {
      v_out[cv] = in.v[cv];
      if (j == g.ny) continue;
    }
    const Nbr n = neighbours(g, i, j, k);
    const df p0 = d2df(in.p[n.c]), h0 = phat_df(in.pn, in.pnm1, n.c), r0 = d2df(__ldg(in.rho + n.c));
    auto face = [&](size_t cn, const df& gk) -> df {
      const df b = beta_df(d2df(__ldg(in.rho + cn)), r0, K, rule);
      const df gp = df_subz(p0, d2df(in.p[cn]));
      const df gh = df_subz(h0, phat_df(in.pn, in.pnm1, cn));
      return df_mulz(gk, df_subz(gp, df_mulz(b, gh)));
    };
    if (j > 0) v_out[cv] = df2d(df_subz(d2df(in.v[cv]), face(n.c - nx, K.gy)));
    u_out[n.c] = df2d(df_subz(d2df(in.u[n.c]), face(n.xm, K.gx)));
    w_out[n.c] = df2d(df_subz(d2df(in.w[n.c]), face(n.zm, K.gz)));
  }
}

__global__ void __launch_bounds__(256) k_df_to_d(const df* __restrict__ a, double* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = df2d(a[i]);
}

__global__ void k_refine_check(DevScalars* sc, int smax, int off, cudaGraphConditionalHandle handle,
                               int use_handle) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  const int cont = refine_decide(sc, smax, off);
  if (use_handle) cudaGraphSetConditional(handle, cont);
}

__global__ void __launch_bounds__(256, 4) k_correct_check(GridDev g, const df* __restrict__ upre,
                                                       const df* __restrict__ vpre, const df* __restrict__ wpre,
                                                       const df* __restrict__ pdf, const df* __restrict__ fdf,
                                                       DevScalars* sc) {
  pdl_enter();
  correct_check_tile(g, upre, vpre, wpre, pdf, fdf, sc, blockIdx.x, gridDim.x);
}

__global__ void k_make_const(GridDev g, DevScalars* sc, double dt) {
  pdl_enter();
  if (threadIdx.x == 0) sc->K = make_const(g, read_rho0(sc), dt);
}

__global__ void k_set_rho0(DevScalars* sc, double rho0) {
  if (threadIdx.x == 0) sc->rho0_bits = (unsigned long long)__double_as_longlong(rho0);
}

// Eq. (31): S = -(1 - C) comp_g - C comp_l + mdot (1/rho_g - 1/rho_l) in pairs;
// zero in under-resolved interface cells (mask set, 0 < C < 1); the one-fluid
// density rho = rho_g (1 - C) + rho_l C when rho is given.  C's range tests
// run on the FP64 bit pattern (C >= 0).
__global__ void __launch_bounds__(256) k_div_constraint(size_t n, const double* __restrict__ C,
                                                        const double* __restrict__ comp_g,
                                                        const double* __restrict__ comp_l,
                                                        const double* __restrict__ mdot,
                                                        const double* __restrict__ rho_g,
                                                        const double* __restrict__ rho_l,
                                                        const unsigned char* __restrict__ mask, double* S,
                                                        double* rho) {
  const df one = {1.0f, 0.0f};
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const double cd = __ldg(C + c);
    const df vc = d2df(cd);
    const df rg = d2df(__ldg(rho_g + c)), rl = d2df(__ldg(rho_l + c));
    const df omc = df_subz(one, vc);  // 1 - C
    const df s = df_addz(df_subz(df_neg(df_mulz(omc, d2df(__ldg(comp_g + c)))), df_mulz(vc, d2df(__ldg(comp_l + c)))),
                         df_mulz(d2df(__ldg(mdot + c)), df_subz(df_recip(rg), df_recip(rl))));
    const unsigned long long cb = (unsigned long long)__double_as_longlong(cd);
    const bool interface_cell = cb > 0ull && cb < 0x3FF0000000000000ull;  // 0 < C < 1
    S[c] = (mask && mask[c] && interface_cell) ? 0.0 : df2d(s);
    if (rho) rho[c] = df2d(df_addz(df_mulz(rg, omc), df_mulz(rl, vc)));
  }
}

namespace {
unsigned grid_for(size_t total, size_t cap) {
  size_t b = (total + 255) / 256;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (unsigned)b;
}
// One wave of 256-thread CTAs: the SMs times the CTAs of `kernel` resident per
// SM (taken once per kernel).  The grid-stride correction kernels launched
// this way keep every resident slot busy to the end; several waves of short
// CTAs measured slower (230 against 216 us at 256^3 for the correction check:
// the slots refill unevenly between waves).
template <auto kernel>
size_t one_wave() {
  static const size_t ctas = [] {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      return (size_t)152 * 4;
    }
    return (size_t)sms * (size_t)per_sm;
  }();
  return ctas;
}
}  // namespace

cudaError_t launch_div_constraint(size_t n, const double* C, const double* comp_g, const double* comp_l,
                                  const double* mdot, const double* rho_g, const double* rho_l,
                                  const unsigned char* mask, double* S, double* rho, cudaStream_t st) {
  k_div_constraint<<<grid_for(n, (size_t)152 * 16), 256, 0, st>>>(n, C, comp_g, comp_l, mdot, rho_g, rho_l, mask, S,
                                                                  rho);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, cudaStream_t st,
                                double* out_p, double* out_u, double* out_v, double* out_w) {
  launch_pdl(k_init_scalars, 1, 32, 0, st, sc, rho0, tol, keep_rho0, out_p, out_u, out_v, out_w);
  return cudaGetLastError();
}

cudaError_t launch_set_rho0(DevScalars* sc, double rho0, cudaStream_t st) {
  k_set_rho0<<<1, 32, 0, st>>>(sc, rho0);
  return cudaGetLastError();
}

cudaError_t launch_make_const(const GridDev& g, DevScalars* sc, double dt, cudaStream_t st) {
  launch_pdl(k_make_const, 1, 32, 0, st, g, sc, dt);
  return cudaGetLastError();
}

cudaError_t launch_rho_min(const double* rho, size_t n, DevScalars* sc, cudaStream_t st) {
  launch_pdl(k_rho_min, grid_for(n, 152 * 8), 256, 0, st, rho, n, sc);
  return cudaGetLastError();
}

cudaError_t launch_correct_pre(const GridDev& g, double dt, const df* upre, const df* vpre, const df* wpre,
                               const df* pdf, double* p64, const DevScalars* sc, double* u_out, double* v_out,
                               double* w_out, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  k_correct_pre<<<grid_for(total, one_wave<k_correct_pre>()), 256, 0, st>>>(g, dt, upre, vpre, wpre, pdf, p64, sc, u_out,
                                                                   v_out, w_out);
  return cudaGetLastError();
}

cudaError_t launch_correct_full(const GridDev& g, const StencilIn& in, const DevScalars* sc, double* u_out,
                                double* v_out, double* w_out, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  k_correct_full<<<grid_for(total, one_wave<k_correct_full>()), 256, 0, st>>>(g, in, sc, u_out, v_out, w_out);
  return cudaGetLastError();
}

cudaError_t launch_correct_check(const GridDev& g, const df* upre, const df* vpre, const df* wpre, const df* pdf,
                                 const df* fdf, DevScalars* sc, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  launch_pdl(k_correct_check, grid_for(total, one_wave<k_correct_check>()), 256, 0, st, g, upre, vpre, wpre, pdf, fdf, sc);
  return cudaGetLastError();
}

cudaError_t launch_df_to_d(const df* a, double* out, size_t n, cudaStream_t st) {
  k_df_to_d<<<grid_for(n, (size_t)152 * 32), 256, 0, st>>>(a, out, n);
  return cudaGetLastError();
}

cudaError_t launch_refine_check(DevScalars* sc, int smax, int off, cudaGraphConditionalHandle handle,
                                int use_handle, cudaStream_t st) {
  launch_pdl(k_refine_check, 1, 32, 0, st, sc, smax, off, handle, use_handle);
  return cudaGetLastError();
}

}  // namespace ppe
