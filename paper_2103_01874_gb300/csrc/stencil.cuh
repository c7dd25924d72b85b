// Finite-volume operators of the uniform staggered (MAC) mesh used by the
// split pressure-gradient projection (Sec. 5 of the paper: velocities on face
// centres, pressure and density at cell centres; Eqs. (32)-(34)), in pair
// (double-float) arithmetic.
//
//   G q on the x face i      = (q_i - q_{i-1}) / dx          periodic in x, z
//   G q on the y face j      = (q_j - q_{j-1}) / dy,  0 on the walls j = 0, ny
//   D a at cell (i,j,k)      = (a_{i+1} - a_i)/dx + (b_{j+1} - b_j)/dy + (c_{k+1} - c_k)/dz
//   L = D G                  the 7-point Laplacian with homogeneous Neumann walls
//   rho_f                    0.5 (rho_L + rho_R) (arithmetic) or 2/(1/rho_L + 1/rho_R)
//   beta_f = 1 - rho_0/rho_f the coefficient of the explicit split term, Eq. (34)
#pragma once
#include "dfloat.cuh"
#include "ppe_internal.h"

namespace ppe {

__device__ __forceinline__ double read_rho0(const DevScalars* sc) {
  return __longlong_as_double((long long)sc->rho0_bits);
}

// Stencil constants (struct StencilConst in ppe_internal.h) from rho_0 and dt:
// the only FP64 arithmetic of a call besides the boundary conversions, done
// once by one thread (k_make_const).
__device__ __forceinline__ StencilConst make_const(const GridDev& g, double rho0, double dt) {
  StencilConst K;
  K.c = d2df(rho0 / dt);
  K.g = d2df(dt / rho0);
  K.r0h = d2df(0.5 * rho0);
  K.r02 = d2df(2.0 * rho0);
  K.idx = d2df(g.idx);
  K.idy = d2df(g.idy);
  K.idz = d2df(g.idz);
  K.gx = d2df(dt / rho0 * g.idx);
  K.gy = d2df(dt / rho0 * g.idy);
  K.gz = d2df(dt / rho0 * g.idz);
  K.lx = d2df(g.idx * g.idx);
  K.ly = d2df(g.idy * g.idy);
  K.lz = d2df(g.idz * g.idz);
  K.cx = d2df(rho0 / dt / g.idx);
  K.cy = d2df(rho0 / dt / g.idy);
  K.cz = d2df(rho0 / dt / g.idz);
  return K;
}

// beta_f = 1 - rho_0 / rho_f for the face between cells with densities a, b
// (unnormalised pair; see the lazy operations in dfloat.cuh)
__device__ __forceinline__ df beta_df(df a, df b, const StencilConst& K, int rule) {
  const df one = {1.0f, 0.0f};
  if (rule == 0) return df_subz(one, df_mulz(K.r02, df_recipz(df_addz(a, b))));   // 1 - 2 rho_0/(a+b)
  return df_subz(one, df_mulz(K.r0h, df_addz(df_recipz(a), df_recipz(b))));        // 1 - (rho_0/2)(1/a+1/b)
}

// Split flux of one face without the 1/h factor, Q~ = beta_f (p_hat_R - p_hat_L)
// + (rho_0/dt) h u*_f, and the explicitly split velocity
// u_pre = u*_f + (dt/rho_0)(1/h) beta_f (p_hat_R - p_hat_L); h the spacing of
// the face's direction, ch = (rho_0/dt) h, gh = (dt/rho_0)/h.  Since
// ch gh = 1, u_pre = gh Q~: one product of the flux instead of a product and
// a sum (the two differ by the pair rounding of the constants, ~1e-14
// relative, and D u_pre = (dt/rho_0)(f + (rho_0/dt) S) holds either way).
// Both are left unnormalised (see the lazy operations in dfloat.cuh): every
// consumer -- the divergence, the correction's subtraction and its exact
// conversion to FP64 -- takes them through lazy pair operations, and a
// normalisation only rewrites the same value (about 5 % fewer instructions
// in the right-hand-side kernels).
struct FaceOut {
  df q, upre;
};
__device__ __forceinline__ FaceOut face_q(df rl, df rh, df pl, df ph, df us, df ch, df gh, const StencilConst& K,
                                          int rule) {
  const df bg = df_mulz(beta_df(rl, rh, K, rule), df_subz(ph, pl));
  FaceOut o;
  o.q = df_addz(bg, df_mulz(ch, us));
  o.upre = df_mulz(gh, o.q);
  return o;
}

// p_hat = 2 p^n - p^{n-1} (Eq. (32)): one FP64 fused multiply-add (a single
// rounding, on the FP64 pipe, which these kernels leave otherwise idle), then
// one split into a pair
__device__ __forceinline__ df phat_of(double pn, double pnm1) { return d2df(fma(2.0, pn, -pnm1)); }

__device__ __forceinline__ df phat_df(const double* pn, const double* pnm1, size_t c) {
  return phat_of(__ldg(pn + c), __ldg(pnm1 + c));
}

struct Nbr {
  size_t c, xp, xm, zp, zm;
};

__device__ __forceinline__ Nbr neighbours(const GridDev& g, int i, int j, int k) {
  Nbr n;
  const size_t nx = (size_t)g.nx, ny = (size_t)g.ny;
  const int ip = (i + 1 == g.nx) ? 0 : i + 1;
  const int im = (i == 0) ? g.nx - 1 : i - 1;
  const int kp = (k + 1 == g.nz) ? 0 : k + 1;
  const int km = (k == 0) ? g.nz - 1 : k - 1;
  n.c = ((size_t)k * ny + j) * nx + i;
  n.xp = n.c - i + ip;
  n.xm = n.c - i + im;
  n.zp = ((size_t)kp * ny + j) * nx + i;
  n.zm = ((size_t)km * ny + j) * nx + i;
  return n;
}

__device__ __forceinline__ void block_max_to(unsigned long long* slot, float v) {
  // v >= 0; reduce over the warp in FP32, one FP64 atomic per warp with a
  // non-zero maximum (all lanes must call).  The maxima only steer the
  // refinement stop test and the reports, so the float hi part suffices.
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0f) atomicMax(slot, (unsigned long long)__double_as_longlong((double)v));
}

// Reduction of two per-thread pair values over the CTA (a fixed shuffle tree,
// then the warps in index order); thread 0 stores the pair of totals in *out.
// Every thread of the CTA must call it (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ void block_pair_sums(df a, df b, double2* out) {
  __shared__ df red_s[2][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = df_norm(a);
  b = df_norm(b);
  for (int o = 16; o > 0; o >>= 1) {
    a = df_add(a, {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)});
    b = df_add(b, {__shfl_down_sync(0xffffffffu, b.hi, o), __shfl_down_sync(0xffffffffu, b.lo, o)});
  }
  if (lane == 0) {
    red_s[0][wid] = a;
    red_s[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = red_s[0][0];
    b = red_s[1][0];
    for (int w = 1; w < nw; ++w) {
      a = df_add(a, red_s[0][w]);
      b = df_add(b, red_s[1][w]);
    }
    *out = make_double2(df2d(a), df2d(b));
  }
}

// Sum of part[0..n) in an order that depends only on n and blockDim.x (thread
// t takes t, t + blockDim.x, ... in turn; then a fixed shuffle and warp tree).
// Every thread of the CTA must call it; thread 0 gets the totals.
__device__ __forceinline__ void sum_parts_fixed(const double2* part, int n, double* tx, double* ty) {
  __shared__ double red_p[2][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double x = 0.0, y = 0.0;
  // each thread adds its entries i = threadIdx.x + m blockDim.x in order of m;
  // eight loads are issued before their additions (the order is unchanged)
  constexpr int U = 8;
  for (int i0 = threadIdx.x; i0 < n; i0 += U * blockDim.x) {
    double2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < n ? __ldcg(part + i) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n) {
        x += v[u].x;
        y += v[u].y;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  if (lane == 0) {
    red_p[0][wid] = x;
    red_p[1][wid] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    x = red_p[0][0];
    y = red_p[1][0];
    for (int w = 1; w < nw; ++w) {
      x += red_p[0][w];
      y += red_p[1][w];
    }
    *tx = x;
    *ty = y;
  }
}

// Totals of the per-CTA partial sums of the current call, formed by one CTA
// (all threads) in a kernel that runs after their producers (the kernel
// boundary orders the accesses): the sum of f from the forward x transform
// (sum_parts_fixed over its CTAs) and the wall flux from the wall tiles of
// k_rhs_march (chunk by chunk, lower wall then upper wall).
__device__ __forceinline__ void finish_sums(DevScalars* sc, const GridDev& g) {
  const size_t nynz = (size_t)g.ny * g.nz;
  const int xp = sc->x_parts;
  const int pp = sc->p_parts;
  double fs = 0.0, ps = 0.0, unused;
  if (xp > 0) sum_parts_fixed(sc->part + nynz, xp, &fs, &unused);
  __syncthreads();  // thread 0 has read the first reduction's shared scratch
  // the sum of the p the last inverse x transform formed: the next correction's
  // zero mode is -sum(p)/ny, which adds -mean(p) to p after the inverse transforms
  // (DCT-III unscaled in its zero mode, z and x inverses scaled by 1/(nx nz))
  if (pp > 0) sum_parts_fixed(sc->part + 2 * nynz, pp, &ps, &unused);
  if (threadIdx.x != 0) return;
  if (pp > 0) {
    sc->zmode = -ps / (double)g.ny;
    sc->p_parts = 0;
  }
  const int nt = sc->rhs_tiles, nc = sc->rhs_chunks;
  if (nt > 0) {
    double ws = 0.0;
    for (int c = 0; c < nc; ++c) {
      ws += sc->part[(size_t)c * nt].x;
      if (nt > 1) ws += sc->part[(size_t)c * nt + nt - 1].x;
    }
    sc->wall_flux = ws;
    sc->rhs_ran = 1;
  }
  if (xp > 0) {
    // A mean below 2^-40 ||f||_inf is rounding noise of a compatible right-hand
    // side (its last bits depend on how the cells were grouped into CTAs); it is
    // not subtracted, which keeps the refinement's result independent of the
    // tile shapes.
    const double mean = fs / ((double)g.nx * (double)g.ny * (double)g.nz);
    const double fmax = __longlong_as_double((long long)sc->fmax_bits);
    sc->f_sum = fs;
    // (an open top has no zero mode: nothing is dropped, nothing left out)
    sc->f_mean = (!g.top_open && fabs(mean) > 0x1p-40 * fmax) ? d2df(mean) : df{0.0f, 0.0f};
    sc->f_ran = 1;
  }
}

}  // namespace ppe
