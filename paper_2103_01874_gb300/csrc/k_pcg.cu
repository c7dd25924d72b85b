// The unsplit projection, Eqs. (29)-(30): the variable-coefficient pressure
// equation
//
//   A p = D[(1/rho_f) G p] = (D u* - S) / dt,       u^{n+1} = u* - dt G p / rho_f,
//
// solved by preconditioned conjugate gradients on K = -A (symmetric positive
// semi-definite; its null space, the constants, is removed by working with
// zero-mean vectors).  The preconditioner is the plan's constant-coefficient
// FFT solve of Eq. (34)'s operator L = D G (z = -L^{-1} r; the solve drops the
// zero mode).  Because that solve runs in FP32 in the refinement form, the
// Polak-Ribiere form of the update is used:
//   beta = z_new . (r_new - r_old) / (z_old . r_old) = -alpha (z_new . K p) / rz_old,
// which tolerates a preconditioner that is not exactly linear.  This is the
// iterative baseline that the split method of Eq. (34) replaces.
//
// Vectors are float pairs (dfloat.cuh); K uses per-face coefficients
// a_f = 1 / (rho_f h^2) formed once per call.  Dot products are reduced per
// CTA in pairs and totalled in a fixed order by one-CTA scalar kernels.
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

namespace {

struct CellIdx {
  uint32_t c, i, j, k;
};

__device__ __forceinline__ CellIdx cell_of(const GridDev& g, uint32_t c) {
  const uint32_t r = fdiv(c, g.fd_nx);  // k ny + j
  const uint32_t k = fdiv(r, g.fd_ny);
  return {c, c - r * (uint32_t)g.nx, r - k * (uint32_t)g.ny, k};
}

// 1 / (rho_f h^2) of the face between cells of densities a, b
template <int RULE>
__device__ __forceinline__ df face_coef(df a, df b, df ih2) {
  if (RULE == 0) return df_mul(df_ldexp2(ih2), df_recip(df_add(a, b)));   // rho_f = (a + b)/2
  return df_mul(df_mul_f(ih2, 0.5f), df_add(df_recip(a), df_recip(b)));   // 1/rho_f = (1/a + 1/b)/2
}

}  // namespace

// Face coefficients, the right side g = (S - D u*)/dt of K p = g (into r), the
// sum of g (per-CTA partials) and max |g|.
template <int RULE>
__global__ void __launch_bounds__(256) k_vc_setup(GridDev g, const double* __restrict__ u,
                                                  const double* __restrict__ v, const double* __restrict__ w,
                                                  const double* __restrict__ S, const double* __restrict__ rho,
                                                  VcConst C, df* ax, df* ay, df* az, df* r, DevScalars* sc,
                                                  double2* part) {
  const uint32_t nx = g.nx, ny = g.ny, nz = g.nz, plane = nx * ny, n = plane * nz;
  df gsum = {0.0f, 0.0f};
  float gmax = 0.0f;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const CellIdx q = cell_of(g, c);
    const uint32_t xm = (q.i == 0) ? c + nx - 1 : c - 1, xp = (q.i + 1 == nx) ? c + 1 - nx : c + 1;
    const uint32_t zm = (q.k == 0) ? c + (nz - 1) * plane : c - plane;
    const uint32_t zp = (q.k + 1 == nz) ? c - (nz - 1) * plane : c + plane;
    const df rc = d2df(__ldg(rho + c));
    ax[c] = face_coef<RULE>(d2df(__ldg(rho + xm)), rc, C.ix2);
    az[c] = face_coef<RULE>(d2df(__ldg(rho + zm)), rc, C.iz2);
    ay[c] = (q.j == 0) ? df{0.0f, 0.0f} : face_coef<RULE>(d2df(__ldg(rho + c - nx)), rc, C.iy2);  // wall: no flux
    const uint32_t cv = (q.k * (ny + 1) + q.j) * nx + q.i;  // v face below the cell
    const df du = df_addz(df_addz(df_mulz(df_sub(d2df(__ldg(u + xp)), d2df(__ldg(u + c))), C.idx),
                                  df_mulz(df_sub(d2df(__ldg(v + cv + nx)), d2df(__ldg(v + cv))), C.idy)),
                          df_mulz(df_sub(d2df(__ldg(w + zp)), d2df(__ldg(w + c))), C.idz));
    const df gv = df_norm(df_mulz(df_subz(d2df(__ldg(S + c)), du), C.idt));
    r[c] = gv;
    gsum = df_addz(gsum, gv);
    gmax = fmaxf(gmax, fabsf(gv.hi));
  }
  block_max_to(&sc->pcg_gmax_bits, gmax);
  block_pair_sums(gsum, df{0.0f, 0.0f}, part + blockIdx.x);
}

// One CTA: mean of g, and the iteration state.
__global__ void k_vc_start(GridDev g, DevScalars* sc, const double2* part, int nparts, double tol, int max_iter) {
  double gs, unused;
  sum_parts_fixed(part, nparts, &gs, &unused);
  if (threadIdx.x != 0) return;
  const double gmean = gs / ((double)g.nx * (double)g.ny * (double)g.nz);
  sc->pcg_gmean = gmean;
  sc->pcg_gmean_df = d2df(gmean);
  sc->pcg_tol = tol;
  sc->pcg_max = max_iter;
  sc->pcg_iter = 0;
  sc->pcg_rz = 0.0;
  sc->pcg_alpha = 0.0;
  sc->pcg_beta = 0.0;
  sc->pcg_rel = 1.0;
  sc->pcg_rmax_bits = 0ull;
  sc->pcg_cont = 1;
}

// Kp = K p and the CTA's part of p . Kp
__global__ void __launch_bounds__(256) k_vc_apply(GridDev g, const df* __restrict__ p, const df* __restrict__ ax,
                                                  const df* __restrict__ ay, const df* __restrict__ az, df* Kp,
                                                  double2* part) {
  const uint32_t nx = g.nx, ny = g.ny, nz = g.nz, plane = nx * ny, n = plane * nz;
  df dot = {0.0f, 0.0f};
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const CellIdx q = cell_of(g, c);
    const uint32_t xm = (q.i == 0) ? c + nx - 1 : c - 1, xp = (q.i + 1 == nx) ? c + 1 - nx : c + 1;
    const uint32_t zm = (q.k == 0) ? c + (nz - 1) * plane : c - plane;
    const uint32_t zp = (q.k + 1 == nz) ? c - (nz - 1) * plane : c + plane;
    const df pc = p[c];
    // sum over the faces of a_f (p_c - p_nbr); the wall faces carry no flux
    df acc = df_mulz(ax[c], df_subz(pc, p[xm]));
    acc = df_addz(acc, df_mulz(ax[xp], df_subz(pc, p[xp])));
    acc = df_addz(acc, df_mulz(az[c], df_subz(pc, p[zm])));
    acc = df_addz(acc, df_mulz(az[zp], df_subz(pc, p[zp])));
    if (q.j > 0) acc = df_addz(acc, df_mulz(ay[c], df_subz(pc, p[c - nx])));
    if (q.j + 1 < ny) acc = df_addz(acc, df_mulz(ay[c + nx], df_subz(pc, p[c + nx])));
    const df kp = df_norm(acc);
    Kp[c] = kp;
    dot = df_addz(dot, df_mulz(pc, kp));
  }
  block_pair_sums(dot, df{0.0f, 0.0f}, part + blockIdx.x);
}

// One CTA: alpha = rz / (p . K p)
__global__ void k_vc_alpha(DevScalars* sc, const double2* part, int nparts) {
  double pkp, unused;
  sum_parts_fixed(part, nparts, &pkp, &unused);
  if (threadIdx.x != 0) return;
  sc->pcg_alpha = (pkp > 0.0 && sc->pcg_rz > 0.0) ? sc->pcg_rz / pkp : 0.0;
}

// x += alpha p, r -= alpha Kp; max |r - mean(g)| (r keeps the mean of g, which
// K p and the solve do not change)
__global__ void __launch_bounds__(256) k_vc_update(uint32_t n, df* x, df* r, const df* __restrict__ p,
                                                   const df* __restrict__ Kp, DevScalars* sc) {
  const df a = d2df(sc->pcg_alpha);
  const df gm = sc->pcg_gmean_df;
  float rmax = 0.0f;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    x[c] = df_norm(df_addz(x[c], df_mulz(a, p[c])));
    const df rn = df_norm(df_subz(r[c], df_mulz(a, Kp[c])));
    r[c] = rn;
    rmax = fmaxf(rmax, fabsf(df_to_f(df_subz(rn, gm))));
  }
  block_max_to(&sc->pcg_rmax_bits, rmax);
}

// The CTA's parts of r . z and z . K p, with z = -zs (zs = L^{-1} r from the
// FFT solve)
__global__ void __launch_bounds__(256) k_vc_dots(uint32_t n, const df* __restrict__ r, const df* __restrict__ zs,
                                                 const df* __restrict__ Kp, double2* part) {
  df d1 = {0.0f, 0.0f}, d2 = {0.0f, 0.0f};
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const df z = zs[c];
    d1 = df_addz(d1, df_mulz(r[c], z));
    d2 = df_addz(d2, df_mulz(z, Kp[c]));
  }
  block_pair_sums(df_neg(d1), df_neg(d2), part + blockIdx.x);
}

// One CTA: beta (0 on the first call), rz, convergence test; sets the WHILE
// condition of the iteration graph when use_handle.
__global__ void k_vc_beta(DevScalars* sc, const double2* part, int nparts, int first,
                          cudaGraphConditionalHandle handle, int use_handle) {
  double rz, zkp;
  sum_parts_fixed(part, nparts, &rz, &zkp);
  if (threadIdx.x != 0) return;
  const double gmax = sc->pcg_gmax_bits ? __longlong_as_double((long long)sc->pcg_gmax_bits) : 0.0;
  double beta = 0.0;
  if (!first) {
    beta = (sc->pcg_rz > 0.0) ? -sc->pcg_alpha * zkp / sc->pcg_rz : 0.0;
    sc->pcg_iter += 1;
    const double rmax = sc->pcg_rmax_bits ? __longlong_as_double((long long)sc->pcg_rmax_bits) : 0.0;
    sc->pcg_rel = gmax > 0.0 ? rmax / gmax : 0.0;
  }
  sc->pcg_rmax_bits = 0ull;
  sc->pcg_beta = beta;
  sc->pcg_rz = rz;
  const int cont = !(sc->pcg_rel <= sc->pcg_tol) && sc->pcg_iter < sc->pcg_max && rz > 0.0 && gmax > 0.0;
  sc->pcg_cont = cont;
  if (use_handle) cudaGraphSetConditional(handle, cont ? 1u : 0u);
}

// p = z + beta p = beta p - zs
__global__ void __launch_bounds__(256) k_vc_pupdate(uint32_t n, df* p, const df* __restrict__ zs,
                                                    const DevScalars* sc) {
  const df b = d2df(sc->pcg_beta);
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    p[c] = df_norm(df_subz(df_mulz(b, p[c]), zs[c]));
}

// The CTA's part of sum x; then one CTA forms the mean.  The FFT preconditioner
// drops the zero mode in its own precision, so x can pick up a small constant
// (FP32: ~1e-8 of max |x|); p is returned with zero mean, as Eq. (30) fixes
// p only up to a constant.
__global__ void __launch_bounds__(256) k_vc_sum(uint32_t n, const df* __restrict__ x, double2* part) {
  df s = {0.0f, 0.0f};
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) s = df_addz(s, x[c]);
  block_pair_sums(s, df{0.0f, 0.0f}, part + blockIdx.x);
}

__global__ void k_vc_xmean(DevScalars* sc, const double2* part, int nparts, double n) {
  double xs, unused;
  sum_parts_fixed(part, nparts, &xs, &unused);
  if (threadIdx.x == 0) sc->pcg_xmean_df = d2df(xs / n);
}

// u^{n+1} = u* - dt G p / rho_f (Eq. (29)) with dt (1/rho_f)/h = dt h a_f; p as
// FP64 with the mean of x removed
__global__ void __launch_bounds__(256) k_vc_correct(GridDev g, const double* __restrict__ u,
                                                    const double* __restrict__ v, const double* __restrict__ w,
                                                    const df* __restrict__ x, const df* __restrict__ ax,
                                                    const df* __restrict__ ay, const df* __restrict__ az, VcConst C,
                                                    const DevScalars* sc, double* p_out, double* u_out,
                                                    double* v_out, double* w_out) {
  const uint32_t nx = g.nx, ny = g.ny, nz = g.nz, plane = nx * ny;
  const df xm0 = sc->pcg_xmean_df;
  const uint32_t total = nz * (ny + 1) * nx;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const uint32_t rr = fdiv(t, g.fd_nx);
    const uint32_t i = t - rr * nx;
    const uint32_t k = fdiv(rr, g.fd_nyp1);
    const uint32_t j = rr - k * (ny + 1);
    const double vt = __ldg(v + t);
    if (j == ny) {  // upper wall: unchanged
      v_out[t] = vt;
      continue;
    }
    const uint32_t c = k * plane + j * nx + i;
    const uint32_t xm = (i == 0) ? c + nx - 1 : c - 1;
    const uint32_t zm = (k == 0) ? c + (nz - 1) * plane : c - plane;
    const df xc = x[c];
    v_out[t] = (j == 0) ? vt : df2d(df_subz(d2df(vt), df_mulz(df_mulz(C.dthy, ay[c]), df_subz(xc, x[c - nx]))));
    u_out[c] = df2d(df_subz(d2df(__ldg(u + c)), df_mulz(df_mulz(C.dthx, ax[c]), df_subz(xc, x[xm]))));
    w_out[c] = df2d(df_subz(d2df(__ldg(w + c)), df_mulz(df_mulz(C.dthz, az[c]), df_subz(xc, x[zm]))));
    p_out[c] = df2d(df_sub(xc, xm0));
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace {
unsigned flat_grid(size_t n) {
  size_t b = (n + 255) / 256;
  const size_t cap = (size_t)152 * 8;
  if (b > cap) b = cap;
  return (unsigned)(b ? b : 1);
}
}  // namespace

unsigned vc_grid(size_t n) { return flat_grid(n); }

cudaError_t launch_vc_setup(const GridDev& g, int rule, const double* u, const double* v, const double* w,
                            const double* S, const double* rho, const VcConst& C, df* ax, df* ay, df* az, df* r,
                            DevScalars* sc, double2* part, cudaStream_t st) {
  const unsigned grid = flat_grid((size_t)g.nx * g.ny * g.nz);
  if (rule == 0)
    k_vc_setup<0><<<grid, 256, 0, st>>>(g, u, v, w, S, rho, C, ax, ay, az, r, sc, part);
  else
    k_vc_setup<1><<<grid, 256, 0, st>>>(g, u, v, w, S, rho, C, ax, ay, az, r, sc, part);
  return cudaGetLastError();
}

cudaError_t launch_vc_start(const GridDev& g, DevScalars* sc, const double2* part, double tol, int max_iter,
                            cudaStream_t st) {
  const int nparts = (int)flat_grid((size_t)g.nx * g.ny * g.nz);
  k_vc_start<<<1, 256, 0, st>>>(g, sc, part, nparts, tol, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_vc_apply(const GridDev& g, const df* p, const df* ax, const df* ay, const df* az, df* Kp,
                            double2* part, cudaStream_t st) {
  k_vc_apply<<<flat_grid((size_t)g.nx * g.ny * g.nz), 256, 0, st>>>(g, p, ax, ay, az, Kp, part);
  return cudaGetLastError();
}

cudaError_t launch_vc_alpha(const GridDev& g, DevScalars* sc, const double2* part, cudaStream_t st) {
  k_vc_alpha<<<1, 256, 0, st>>>(sc, part, (int)flat_grid((size_t)g.nx * g.ny * g.nz));
  return cudaGetLastError();
}

cudaError_t launch_vc_update(const GridDev& g, df* x, df* r, const df* p, const df* Kp, DevScalars* sc,
                             cudaStream_t st) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  k_vc_update<<<flat_grid(n), 256, 0, st>>>((uint32_t)n, x, r, p, Kp, sc);
  return cudaGetLastError();
}

cudaError_t launch_vc_dots(const GridDev& g, const df* r, const df* zs, const df* Kp, double2* part,
                           cudaStream_t st) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  k_vc_dots<<<flat_grid(n), 256, 0, st>>>((uint32_t)n, r, zs, Kp, part);
  return cudaGetLastError();
}

cudaError_t launch_vc_beta(const GridDev& g, DevScalars* sc, const double2* part, int first,
                           cudaGraphConditionalHandle handle, int use_handle, cudaStream_t st) {
  k_vc_beta<<<1, 256, 0, st>>>(sc, part, (int)flat_grid((size_t)g.nx * g.ny * g.nz), first, handle, use_handle);
  return cudaGetLastError();
}

cudaError_t launch_vc_pupdate(const GridDev& g, df* p, const df* zs, const DevScalars* sc, cudaStream_t st) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  k_vc_pupdate<<<flat_grid(n), 256, 0, st>>>((uint32_t)n, p, zs, sc);
  return cudaGetLastError();
}

cudaError_t launch_vc_correct(const GridDev& g, const double* u, const double* v, const double* w, const df* x,
                              const df* ax, const df* ay, const df* az, const VcConst& C, DevScalars* sc,
                              double2* part, double* p_out, double* u_out, double* v_out, double* w_out,
                              cudaStream_t st) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  const unsigned gs = flat_grid(n);
  k_vc_sum<<<gs, 256, 0, st>>>((uint32_t)n, x, part);
  k_vc_xmean<<<1, 256, 0, st>>>(sc, part, (int)gs, (double)n);
  const size_t total = (size_t)g.nx * (g.ny + 1) * g.nz;
  k_vc_correct<<<flat_grid(total), 256, 0, st>>>(g, u, v, w, x, ax, ay, az, C, sc, p_out, u_out, v_out, w_out);
  return cudaGetLastError();
}

}  // namespace ppe
