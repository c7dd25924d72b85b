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
// the face's direction, ch = (rho_0/dt) h, gh = (dt/rho_0)/h.
struct FaceOut {
  df q, upre;
};
__device__ __forceinline__ FaceOut face_q(df rl, df rh, df pl, df ph, df us, df ch, df gh, const StencilConst& K,
                                          int rule) {
  const df bg = df_mulz(beta_df(rl, rh, K, rule), df_subz(ph, pl));
  FaceOut o;
  o.q = df_norm(df_addz(bg, df_mulz(ch, us)));
  o.upre = df_norm(df_addz(us, df_mulz(gh, bg)));
  return o;
}

__device__ __forceinline__ df phat_df(const double* pn, const double* pnm1, size_t c) {
  // p_hat = 2 p^n - p^{n-1}, Eq. (32)
  return df_sub(df_ldexp2(d2df(__ldg(pn + c))), d2df(__ldg(pnm1 + c)));
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
  // v >= 0; reduce over the warp in FP32, one FP64 atomic per warp (all lanes must call).
  // The maxima only steer the refinement stop test, so the float hi part suffices.
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, (unsigned long long)__double_as_longlong((double)v));
}

}  // namespace ppe
