// Device functions of the point-wise passes as functions of the CTA index,
// shared by their own kernels (k_stencil.cu) and the persistent batched kernel
// (k_batch.cu): rho_0 = min(rho) (text after Eq. (32)), the refinement's loop
// decision, and Eq. (33) fused with the residual of the corrected p.
#pragma once
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

// keep_rho0: leave rho_0 as the last right-hand side set it (ppe_solve).
// out_p non-null: also record the ppe_project outputs (read by the fused
// correction check, so that a captured refinement graph serves every call).
__device__ __forceinline__ void init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, double* out_p,
                                             double* out_u, double* out_v, double* out_w) {
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
__device__ __forceinline__ void rho_min_body(const double* __restrict__ rho, size_t n, DevScalars* sc, uint32_t bid,
                                             uint32_t nblk) {
  unsigned long long m = 0x7FF0000000000000ull;
  const size_t stride = (size_t)nblk * blockDim.x;
  for (size_t i0 = bid * (size_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
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

// Test of a residual and the loop decision.
//  off = 0 (probe): slot s = iter holds r after s-1 corrections.  Converged if
//    ||r||_inf <= tol ||f||_inf; else correction s follows if s <= smax.
//  off = 1 (after the fused correction): slot s = iter + 1 holds r after
//    `iter` corrections.  Converged as above; else another correction follows
//    if iter < smax (iter is advanced).
// `sweeps` counts applied corrections; `cont` (and the graph condition) asks
// for another round.
__device__ __forceinline__ int refine_decide(DevScalars* sc, int smax, int off) {
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
  return cont;
}


// Eq. (33) from u_pre as in k_correct_pre, with p as pairs, plus the residual
// r = f - L p of that same p at every cell (max into rmax[iter + 1]), so that the
// convergence test after a correction needs no separate pass.
// SUB: the mean of f is non-zero and is left out of the residual (the solve drops it)
// OPEN: outflow top (the top face is corrected, the top cells see the ghost -p)
template <bool SUB, bool OPEN>
__device__ __forceinline__ void correct_check_body(const GridDev& g, const df* upre,
                                                   const df* vpre, const df* wpre,
                                                   const df* pdf, const df* fdf,
                                                   DevScalars* sc, df fmean, uint32_t bid,
                                                   uint32_t nblk) {
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
  const uint32_t stride = nblk * blockDim.x;
  for (uint32_t t = bid * blockDim.x + threadIdx.x; t < total; t += stride) {
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

// One CTA (index bid of nblk) of the fused correction check.
__device__ __forceinline__ void correct_check_tile(const GridDev& g, const df* upre, const df* vpre, const df* wpre,
                                                   const df* pdf, const df* fdf, DevScalars* sc, uint32_t bid,
                                                   uint32_t nblk) {
  const df fmean = sc->f_mean;
  if (g.top_open)
    correct_check_body<false, true>(g, upre, vpre, wpre, pdf, fdf, sc, fmean, bid, nblk);  // no mean is left out
  else if (fmean.hi == 0.0f)
    correct_check_body<false, false>(g, upre, vpre, wpre, pdf, fdf, sc, fmean, bid, nblk);
  else
    correct_check_body<true, false>(g, upre, vpre, wpre, pdf, fdf, sc, fmean, bid, nblk);
}

}  // namespace ppe
