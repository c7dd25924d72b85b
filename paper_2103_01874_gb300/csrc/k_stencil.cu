// Point-wise kernels of the projection: rho_0 = min(rho) (text after Eq. (32)),
// the velocity correction of Eq. (33), and the device-side refinement control.
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

// keep_rho0: leave rho_0 as the last right-hand side set it (ppe_solve).
// out_p non-null: also record the ppe_project outputs (read by the fused
// correction check, so that a captured refinement graph serves every call).
__global__ void k_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, double* out_p,
                               double* out_u, double* out_v, double* out_w) {
  if (threadIdx.x != 0) return;
  if (out_p) {
    sc->out_p = out_p;
    sc->out_u = out_u;
    sc->out_v = out_v;
    sc->out_w = out_w;
  }
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
  sc->f_sum = 0.0;
  sc->f_mean = {0.0f, 0.0f};
  sc->f_ran = 0;
  sc->x_parts = 0;
  sc->dev_err = 0;
  sc->zmode = 0.0;
  sc->p_parts = 0;
  if (!keep_rho0) {  // a call that assembles f: its compatibility sums start here
    sc->smax_bits = 0ull;
    sc->wallv_bits = 0ull;
    sc->wall_flux = 0.0;
    sc->rhs_ran = 0;
    sc->rhs_tiles = 0;
    sc->rhs_chunks = 0;
  }
}

// rho > 0 (densities), so the IEEE bit patterns order like the values and the
// minimum runs on 64-bit integers (no FP64 instructions); 4 loads in flight.
__global__ void __launch_bounds__(256) k_rho_min(const double* __restrict__ rho, size_t n, DevScalars* sc) {
  unsigned long long m = 0x7FF0000000000000ull;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    unsigned long long b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t i = i0 + u * stride;
      b[u] = (i < n) ? (unsigned long long)__double_as_longlong(__ldg(rho + i)) : 0x7FF0000000000000ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) m = b[u] < m ? b[u] : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
    m = q < m ? q : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMin(&sc->rho0_bits, m);
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

// Test of a residual and the loop decision.
//  off = 0 (probe): slot s = iter holds r after s-1 corrections.  Converged if
//    ||r||_inf <= tol ||f||_inf; else correction s follows if s <= smax.
//  off = 1 (after the fused correction): slot s = iter + 1 holds r after
//    `iter` corrections.  Converged as above; else another correction follows
//    if iter < smax (iter is advanced).
// `sweeps` counts applied corrections; `cont` (and the graph condition) asks
// for another round.
__global__ void k_refine_check(DevScalars* sc, int smax, int off, cudaGraphConditionalHandle handle,
                               int use_handle) {
  if (threadIdx.x != 0) return;
  const int it = sc->iter;
  const int s = it + off;
  const double r = __longlong_as_double((long long)sc->rmax_bits[s]);
  const double f = __longlong_as_double((long long)sc->fmax_bits);
  sc->last_slot = s;
  int cont = 0;
  if (r <= sc->tol * f) {
    sc->done = 1;
    sc->sweeps = s - 1;
  } else if (off == 0 && s <= smax) {
    sc->sweeps = s;
    sc->iter = s + 1;
    cont = 1;
  } else if (off == 1 && it < smax) {
    sc->sweeps = it;
    sc->iter = it + 1;
    cont = 1;
  } else {
    sc->sweeps = (off == 1) ? it : smax;
  }
  sc->cont = cont;
  if (use_handle) cudaGraphSetConditional(handle, cont);
}


// Eq. (33) from u_pre as in k_correct_pre, with p as pairs, plus the residual
// r = f - L p of that same p at every cell (max into rmax[iter + 1]), so that the
// convergence test after a correction needs no separate pass.
// SUB: the mean of f is non-zero and is left out of the residual (the solve drops it)
// OPEN: outflow top (the top face is corrected, the top cells see the ghost -p)
template <bool SUB, bool OPEN>
__device__ __forceinline__ void correct_check_body(const GridDev& g, const df* __restrict__ upre,
                                                   const df* __restrict__ vpre, const df* __restrict__ wpre,
                                                   const df* __restrict__ pdf, const df* __restrict__ fdf,
                                                   DevScalars* sc, df fmean) {
  // 32-bit offsets: grids up to 1024^3 (v: nx (ny+1) nz < 2^32)
  const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny, nz = (uint32_t)g.nz;
  const uint32_t plane = ny * nx;
  const uint32_t total = nz * (ny + 1) * nx;
  const StencilConst K = sc->K;
  double* const u_out = sc->out_u;
  double* const v_out = sc->out_v;
  double* const w_out = sc->out_w;
  double* const p_out = sc->out_p;
  const int slot = sc->iter + 1;
  float vmax = 0.0f;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    // t indexes the v faces [k][j][i], j = 0..ny; j < ny also carries cell (i, j, k)
    const uint32_t r = fdiv(t, g.fd_nx);
    const uint32_t i = t - r * nx;
    const uint32_t k = fdiv(r, g.fd_nyp1);
    const uint32_t j = r - k * (ny + 1);
    const df vp = vpre[t];
    if (j == ny) {  // top face: a wall keeps v; an open top sees the ghost -p of the cell below
      if (OPEN) {
        const df pt = pdf[k * plane + (ny - 1) * nx + i];  // the top cell (i, ny-1, k)
        v_out[t] = df2d(df_subz(vp, df_mulz(K.gy, df_subz(df_neg(pt), pt))));
      } else {
        v_out[t] = df2d(vp);
      }
      continue;
    }
    const uint32_t c = k * plane + j * nx + i;
    const uint32_t xm = (i == 0) ? c + nx - 1 : c - 1;
    const uint32_t xp = (i + 1 == nx) ? c + 1 - nx : c + 1;
    const uint32_t zm = (k == 0) ? c + (nz - 1) * plane : c - plane;
    const uint32_t zp = (k + 1 == nz) ? c - (nz - 1) * plane : c + plane;
    const df up = upre[c], wp = wpre[c], q = pdf[c];
    const df pxm = pdf[xm], pxp = pdf[xp], pzm = pdf[zm], pzp = pdf[zp];
    const df pym = (j > 0) ? pdf[c - nx] : q;
    const df pyp = (j + 1 < ny) ? pdf[c + nx] : (OPEN ? df_neg(q) : q);
    const df fv = fdf[c];
    // backward differences (the faces of this cell) serve Eq. (33) and the residual
    const df dxm = df_subz(q, pxm), dym = df_subz(q, pym), dzm = df_subz(q, pzm);
    v_out[t] = df2d(j == 0 ? vp : df_subz(vp, df_mulz(K.gy, dym)));  // lower wall: v unchanged
    u_out[c] = df2d(df_subz(up, df_mulz(K.gx, dxm)));
    w_out[c] = df2d(df_subz(wp, df_mulz(K.gz, dzm)));
    p_out[c] = df2d(q);
    const df lx = df_subz(df_subz(pxp, q), dxm);
    const df ly = df_subz(df_subz(pyp, q), dym);
    const df lz = df_subz(df_subz(pzp, q), dzm);
    const df lap = df_addz(df_addz(df_mulz(lx, K.lx), df_mulz(ly, K.ly)), df_mulz(lz, K.lz));
    const df fr = SUB ? df_subz(fv, fmean) : fv;
    vmax = fmaxf(vmax, fabsf(df_to_f(df_subz(fr, lap))));
  }
  block_max_to(&sc->rmax_bits[slot], vmax);
}

__global__ void __launch_bounds__(256, 4) k_correct_check(GridDev g, const df* __restrict__ upre,
                                                       const df* __restrict__ vpre, const df* __restrict__ wpre,
                                                       const df* __restrict__ pdf, const df* __restrict__ fdf,
                                                       DevScalars* sc) {
  const df fmean = sc->f_mean;
  if (g.top_open)
    correct_check_body<false, true>(g, upre, vpre, wpre, pdf, fdf, sc, fmean);  // no mean is left out
  else if (fmean.hi == 0.0f)
    correct_check_body<false, false>(g, upre, vpre, wpre, pdf, fdf, sc, fmean);
  else
    correct_check_body<true, false>(g, upre, vpre, wpre, pdf, fdf, sc, fmean);
}

__global__ void k_make_const(GridDev g, DevScalars* sc, double dt) {
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
  k_init_scalars<<<1, 32, 0, st>>>(sc, rho0, tol, keep_rho0, out_p, out_u, out_v, out_w);
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

cudaError_t launch_correct_check(const GridDev& g, const df* upre, const df* vpre, const df* wpre, const df* pdf,
                                 const df* fdf, DevScalars* sc, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  k_correct_check<<<grid_for(total, (size_t)152 * 64), 256, 0, st>>>(g, upre, vpre, wpre, pdf, fdf, sc);
  return cudaGetLastError();
}

cudaError_t launch_df_to_d(const df* a, double* out, size_t n, cudaStream_t st) {
  k_df_to_d<<<grid_for(n, (size_t)152 * 32), 256, 0, st>>>(a, out, n);
  return cudaGetLastError();
}

cudaError_t launch_refine_check(DevScalars* sc, int smax, int off, cudaGraphConditionalHandle handle,
                                int use_handle, cudaStream_t st) {
  k_refine_check<<<1, 32, 0, st>>>(sc, smax, off, handle, use_handle);
  return cudaGetLastError();
}

}  // namespace ppe
