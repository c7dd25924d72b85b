// Point-wise kernels of the projection: rho_0 = min(rho) (text after Eq. (32)),
// the velocity correction of Eq. (33), and the device-side refinement control.
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

// Eq. (33): u^{n+1} = u* - dt [G p / rho_0 + (1/rho_f - 1/rho_0) G p_hat] on
// every face; wall faces of v (j = 0, ny) keep v*.  One thread per (i, j, k)
// with 0 <= j <= ny: it writes the x and z faces of cell (i, j, k) (j < ny)
// and the y face j.
__global__ void __launch_bounds__(256) k_correct(GridDev g, StencilIn in, const DevScalars* sc, double* u_out,
                                                 double* v_out, double* w_out) {
  const size_t nx = (size_t)g.nx, ny = (size_t)g.ny;
  const size_t total = (size_t)g.nz * (ny + 1) * nx;
  const double rho0 = read_rho0(sc), irho0 = 1.0 / rho0, dt = in.dt;
  const int rule = in.face_rule;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % nx);
    const size_t r = t / nx;
    const int j = (int)(r % (ny + 1));
    const int k = (int)(r / (ny + 1));
    const size_t vc = t;  // v index (k*(ny+1) + j)*nx + i
    if (j == 0 || j == g.ny) {
      v_out[vc] = in.v[vc];
    }
    if (j < g.ny) {
      const Nbr n = neighbours(g, i, j, k);
      const double p0 = ldg(in.p + n.c), h0 = phat_at(in, n.c), r0 = ldg(in.rho + n.c);
      if (j > 0) {
        const size_t cy = n.c - nx;
        const double gp = (p0 - ldg(in.p + cy)) * g.idy;
        const double gh = (h0 - phat_at(in, cy)) * g.idy;
        const double ir = inv_face(ldg(in.rho + cy), r0, rule);
        v_out[vc] = in.v[vc] - dt * (gp * irho0 + (ir - irho0) * gh);
      }
      {
        const double gp = (p0 - ldg(in.p + n.xm)) * g.idx;
        const double gh = (h0 - phat_at(in, n.xm)) * g.idx;
        const double ir = inv_face(ldg(in.rho + n.xm), r0, rule);
        u_out[n.c] = in.u[n.c] - dt * (gp * irho0 + (ir - irho0) * gh);
      }
      {
        const double gp = (p0 - ldg(in.p + n.zm)) * g.idz;
        const double gh = (h0 - phat_at(in, n.zm)) * g.idz;
        const double ir = inv_face(ldg(in.rho + n.zm), r0, rule);
        w_out[n.c] = in.w[n.c] - dt * (gp * irho0 + (ir - irho0) * gh);
      }
    }
  }
}

// Before refinement sweep s (1-based; s = smax + 1 is the final measurement):
// stop once ||r||_inf <= tol ||f||_inf.  `sweeps` counts applied corrections.
__global__ void k_refine_check(DevScalars* sc, int s, int smax) {
  if (threadIdx.x != 0 || sc->done) return;
  const double r = __longlong_as_double((long long)sc->rmax_bits[s]);
  const double f = __longlong_as_double((long long)sc->fmax_bits);
  sc->last_slot = s;
  if (r <= sc->tol * f) {
    sc->done = 1;
    sc->sweeps = s - 1;
  } else {
    sc->sweeps = s < smax ? s : smax;
  }
}

__global__ void k_set_rho0(DevScalars* sc, double rho0) {
  if (threadIdx.x == 0) sc->rho0_bits = (unsigned long long)__double_as_longlong(rho0);
}

cudaError_t launch_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, cudaStream_t st) {
  k_init_scalars<<<1, 32, 0, st>>>(sc, rho0, tol, keep_rho0);
  return cudaGetLastError();
}

cudaError_t launch_rho_min(const double* rho, size_t n, DevScalars* sc, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_rho_min<<<blocks, 256, 0, st>>>(rho, n, sc);
  return cudaGetLastError();
}

cudaError_t launch_correct(const GridDev& g, const StencilIn& in, const DevScalars* sc, double* u_out, double* v_out,
                           double* w_out, cudaStream_t st) {
  const size_t total = (size_t)g.nz * (g.ny + 1) * g.nx;
  size_t blocks = (total + 255) / 256;
  if (blocks > (size_t)152 * 64) blocks = (size_t)152 * 64;
  k_correct<<<(unsigned)blocks, 256, 0, st>>>(g, in, sc, u_out, v_out, w_out);
  return cudaGetLastError();
}

cudaError_t launch_refine_check(DevScalars* sc, int sweep, int smax, cudaStream_t st) {
  k_refine_check<<<1, 32, 0, st>>>(sc, sweep, smax);
  return cudaGetLastError();
}

cudaError_t launch_set_rho0(DevScalars* sc, double rho0, cudaStream_t st) {
  k_set_rho0<<<1, 32, 0, st>>>(sc, rho0);
  return cudaGetLastError();
}

}  // namespace ppe
