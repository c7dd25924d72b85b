// Finite-volume operators of the uniform staggered (MAC) mesh used by the
// split pressure-gradient projection (Sec. 5 of the paper: velocities on face
// centres, pressure and density at cell centres; Eqs. (32)-(34)).
//
//   G q on the x face i      = (q_i - q_{i-1}) / dx          periodic in x, z
//   G q on the y face j      = (q_j - q_{j-1}) / dy,  0 on the walls j = 0, ny
//   D a at cell (i,j,k)      = (a_{i+1} - a_i)/dx + (b_{j+1} - b_j)/dy + (c_{k+1} - c_k)/dz
//   L = D G                  the 7-point Laplacian with homogeneous Neumann walls
//   rho_f                    0.5 (rho_L + rho_R) (arithmetic) or 2/(1/rho_L + 1/rho_R)
#pragma once
#include "ppe_internal.h"

namespace ppe {

__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }

__device__ __forceinline__ double phat_at(const StencilIn& in, size_t c) {
  // p_hat = 2 p^n - p^{n-1}, Eq. (32)
  return 2.0 * ldg(in.pn + c) - ldg(in.pnm1 + c);
}

// 1 - rho_0 / rho_f, the coefficient of the explicit split term in Eq. (34)
__device__ __forceinline__ double beta_face(double a, double b, double rho0, int rule) {
  if (rule == 0) return 1.0 - rho0 / (0.5 * (a + b));
  return 1.0 - rho0 * 0.5 * (1.0 / a + 1.0 / b);
}

// 1 / rho_f
__device__ __forceinline__ double inv_face(double a, double b, int rule) {
  if (rule == 0) return 1.0 / (0.5 * (a + b));
  return 0.5 * (1.0 / a + 1.0 / b);
}

struct Nbr {
  size_t c, xp, xm, zp, zm;
  int ip, im, kp, km;
};

__device__ __forceinline__ Nbr neighbours(const GridDev& g, int i, int j, int k) {
  Nbr n;
  const size_t nx = (size_t)g.nx, ny = (size_t)g.ny;
  n.ip = (i + 1 == g.nx) ? 0 : i + 1;
  n.im = (i == 0) ? g.nx - 1 : i - 1;
  n.kp = (k + 1 == g.nz) ? 0 : k + 1;
  n.km = (k == 0) ? g.nz - 1 : k - 1;
  n.c = ((size_t)k * ny + j) * nx + i;
  n.xp = n.c - i + n.ip;
  n.xm = n.c - i + n.im;
  n.zp = ((size_t)n.kp * ny + j) * nx + i;
  n.zm = ((size_t)n.km * ny + j) * nx + i;
  return n;
}

// Eq. (34) right-hand side at cell (i, j, k):
//   f = D[(1 - rho_0/rho_f) G p_hat] + (rho_0/dt)(D u* - S)
__device__ __forceinline__ double rhs_at(const GridDev& g, const StencilIn& in, double rho0, int i, int j,
                                         int k) {
  const Nbr n = neighbours(g, i, j, k);
  const size_t nx = (size_t)g.nx;
  const double h0 = phat_at(in, n.c), r0 = ldg(in.rho + n.c);
  const int rule = in.face_rule;
  // x faces i+1 (right) and i (left)
  double fx = beta_face(r0, ldg(in.rho + n.xp), rho0, rule) * (phat_at(in, n.xp) - h0) -
              beta_face(ldg(in.rho + n.xm), r0, rho0, rule) * (h0 - phat_at(in, n.xm));
  double fy = 0.0;
  if (j + 1 < g.ny) {
    const size_t cy = n.c + nx;
    fy += beta_face(r0, ldg(in.rho + cy), rho0, rule) * (phat_at(in, cy) - h0);
  }
  if (j > 0) {
    const size_t cy = n.c - nx;
    fy -= beta_face(ldg(in.rho + cy), r0, rho0, rule) * (h0 - phat_at(in, cy));
  }
  double fz = beta_face(r0, ldg(in.rho + n.zp), rho0, rule) * (phat_at(in, n.zp) - h0) -
              beta_face(ldg(in.rho + n.zm), r0, rho0, rule) * (h0 - phat_at(in, n.zm));
  const double split = fx * g.idx * g.idx + fy * g.idy * g.idy + fz * g.idz * g.idz;
  const size_t vc = ((size_t)k * (g.ny + 1) + j) * nx + i;
  const double divu = (ldg(in.u + n.xp) - ldg(in.u + n.c)) * g.idx +
                      (ldg(in.v + vc + nx) - ldg(in.v + vc)) * g.idy +
                      (ldg(in.w + n.zp) - ldg(in.w + n.c)) * g.idz;
  return split + rho0 * in.inv_dt * (divu - ldg(in.S + n.c));
}

// r = f - L p at cell (i, j, k)
__device__ __forceinline__ double resid_at(const GridDev& g, const StencilIn& in, int i, int j, int k) {
  const Nbr n = neighbours(g, i, j, k);
  const size_t nx = (size_t)g.nx;
  const double p0 = ldg(in.p + n.c);
  double ly = 0.0;
  if (j + 1 < g.ny) ly += ldg(in.p + n.c + nx) - p0;
  if (j > 0) ly -= p0 - ldg(in.p + n.c - nx);
  const double lap = (ldg(in.p + n.xp) - 2.0 * p0 + ldg(in.p + n.xm)) * (g.idx * g.idx) + ly * (g.idy * g.idy) +
                     (ldg(in.p + n.zp) - 2.0 * p0 + ldg(in.p + n.zm)) * (g.idz * g.idz);
  return ldg(in.f + n.c) - lap;
}

__device__ __forceinline__ double read_rho0(const DevScalars* sc) {
  return __longlong_as_double((long long)sc->rho0_bits);
}

__device__ __forceinline__ void block_max_to(unsigned long long* slot, double v) {
  // v >= 0; reduce over the block, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

}  // namespace ppe
