// Host side of libppe: plans, tables and the C entry points declared in
// include/ppe.h (split pressure-gradient projection, Sec. 5.4 of the paper,
// Eqs. (32)-(34)).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/ppe.h"
#include "ppe_internal.h"

using namespace ppe;

struct ppe_plan_s {
  ppe_grid g;
  ppe_options opt;
  cudaStream_t stream;
  GridDev gd;
  int nxh;
  RadixPlan rp_half;  // nx/2
  RadixPlan rp_z;     // nz
  int lpb;            // lines per CTA in the x passes
  int tkx;            // kx columns per CTA in the z pass
  bool fp32;
  size_t cplx_bytes;
  void* spec;         // cpx<T>[nz][ny][nxh]
  void* tw_x;         // cpx<T>[nx]: exp(-2 pi i t/nx)
  void* tw_z;         // cpx<T>[nz]
  void* tab;          // T: elimination multipliers
  int* line_off;
  int* line_len;
  double a_y;         // 1/dy^2
  double* fbuf;       // FP64 right-hand side kept for the residual (FP32_REFINE)
  DevScalars* sc;
  // ppe_project_host staging (allocated on first use)
  double* io[12];
  size_t workspace;
  // per-kernel CUDA-event records (ppe_profile)
  int prof_on;
  std::vector<cudaEvent_t>* prof_ev;   // pool: 2 events per record
  std::vector<int>* prof_name;         // kernel id per record
  int prof_used;
  int prof_dropped;
};

namespace {

bool is_23_smooth(int n) {
  if (n <= 0) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

bool dim_ok(int n) { return n >= 8 && n <= kMaxDim && is_23_smooth(n); }

RadixPlan radix_plan(int n) {
  RadixPlan rp;
  memset(&rp, 0, sizeof(rp));
  rp.n = n;
  int m = n;
  while (m % 4 == 0) { rp.r[rp.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { rp.r[rp.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { rp.r[rp.nst++] = 3; m /= 3; }
  return rp;
}

// exp(-2 pi i t / n) with the argument reduced to [0, pi/4] before calling
// cos/sin, so that t/n in {0, 1/4, 1/2, 3/4} gives exact values.
void cis_neg(long t, long n, double* re, double* im) {
  t %= n;
  if (t < 0) t += n;
  const long q = (4 * t) / n;        // quadrant
  const long r = 4 * t - q * n;      // angle = (pi/2) (r/n) within the quadrant, r in [0, n)
  double c, s;
  if (2 * r <= n) {
    const double phi = (M_PI / 2) * ((double)r / (double)n);
    c = cos(phi);
    s = sin(phi);
  } else {
    const double phi = (M_PI / 2) * ((double)(n - r) / (double)n);
    c = sin(phi);
    s = cos(phi);
  }
  double cr, sr;  // rotate by q quarter turns: angle + q pi/2
  switch (q) {
    case 0: cr = c; sr = s; break;
    case 1: cr = -s; sr = c; break;
    case 2: cr = -c; sr = -s; break;
    default: cr = s; sr = -c; break;
  }
  *re = cr;
  *im = -sr;
}

// sin(pi t / n)
double sin_pi_frac(long t, long n) {
  double re, im;
  cis_neg(t, 2 * n, &re, &im);
  return -im;
}

// cudaErrorMemoryAllocation -> PPE_ERR_OUT_OF_MEMORY; anything else (no device,
// driver mismatch) -> PPE_ERR_CUDA.
ppe_status alloc_status(cudaError_t e) {
  if (e == cudaSuccess) return PPE_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PPE_ERR_OUT_OF_MEMORY : PPE_ERR_CUDA;
}

template <typename T>
ppe_status upload(void** dst, const std::vector<T>& v) {
  ppe_status s = alloc_status(cudaMalloc(dst, v.size() * sizeof(T)));
  if (s != PPE_OK) return s;
  if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return PPE_ERR_CUDA;
  return PPE_OK;
}

template <typename T>
ppe_status make_twiddles(void** dst, int n) {
  std::vector<cpx<T>> v(n);
  for (int t = 0; t < n; ++t) {
    double re, im;
    cis_neg(t, n, &re, &im);
    v[t].x = (T)re;
    v[t].y = (T)im;
  }
  return upload(dst, v);
}

// Elimination multipliers of the Neumann tridiagonal systems, one per
// (kx, kz) line (see k_ythomas).  Computed in FP64; for FP32 plans rounded.
template <typename T>
ppe_status make_thomas(ppe_plan_t P) {
  const int nx = P->g.nx, ny = P->g.ny, nz = P->g.nz, nxh = P->nxh;
  const double dx = P->g.lx / nx, dy = P->g.ly / ny, dz = P->g.lz / nz;
  const double a = 1.0 / (dy * dy);
  const int lines = nxh * nz;
  std::vector<int> off(lines), len(lines);
  std::vector<T> tab;
  tab.reserve((size_t)lines * 8);
  std::vector<double> m(ny);
  std::vector<T> mt(ny);
  for (int kz = 0; kz < nz; ++kz) {
    const double sz = sin_pi_frac(kz, nz);
    const double lz = -(4.0 / (dz * dz)) * sz * sz;
    for (int kx = 0; kx < nxh; ++kx) {
      const double sx = sin_pi_frac(kx, nx);
      const double lam = -(4.0 / (dx * dx)) * sx * sx + lz;
      const bool zero = (kx == 0 && kz == 0);
      m[0] = zero ? 0.0 : 1.0 / (-a + lam);
      for (int j = 1; j < ny - 1; ++j) m[j] = 1.0 / ((-2.0 * a + lam) - a * (a * m[j - 1]));
      m[ny - 1] = 1.0 / ((-a + lam) - a * (a * m[ny - 2]));
      for (int j = 0; j < ny; ++j) mt[j] = (T)m[j];
      int J = ny - 1;  // entries m_0 .. m_{J-1} stored; m_j == m_{ny-2} for J <= j <= ny-2
      while (J > 0 && mt[J - 1] == mt[ny - 2]) --J;
      const int line = kz * nxh + kx;
      off[line] = (int)tab.size();
      len[line] = J;
      tab.push_back(mt[ny - 2]);
      tab.push_back(mt[ny - 1]);
      for (int j = 0; j < J; ++j) tab.push_back(mt[j]);
    }
  }
  ppe_status s;
  if ((s = upload(&P->tab, tab)) != PPE_OK) return s;
  if ((s = upload((void**)&P->line_off, off)) != PPE_OK) return s;
  if ((s = upload((void**)&P->line_len, len)) != PPE_OK) return s;
  P->workspace += tab.size() * sizeof(T) + 2 * sizeof(int) * (size_t)lines;
  return PPE_OK;
}

int choose_lpb(int nx) {
  int l = 2048 / nx;
  if (l < 1) l = 1;
  if (l > 64) l = 64;
  return l;
}

int choose_tkx(int nz, bool fp32) {
  const size_t cb = fp32 ? 8 : 16;
  int t = fp32 ? 16 : 8;
  while (t > 2 && 2 * cb * (size_t)t * nz > 160 * 1024) t /= 2;
  return t;
}

ppe_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PPE_OK : PPE_ERR_CUDA; }

// Kernel names reported by ppe_profile_read.
enum KernelId { K_INIT, K_RHO_MIN, K_XFWD_RHS, K_XFWD_F, K_XFWD_RESID, K_ZFFT_FWD, K_YTHOMAS, K_ZFFT_INV,
                K_XINV, K_XINV_ACC, K_CORRECT, K_CHECK, K_COUNT };
const char* const kKernelNames[K_COUNT] = {"k_init_scalars", "k_rho_min", "k_xfwd_rhs", "k_xfwd_f",
                                           "k_xfwd_resid", "k_zfft_fwd", "k_ythomas", "k_zfft_inv",
                                           "k_xinv", "k_xinv_accum", "k_correct", "k_refine_check"};
constexpr int kProfMax = 16384;

int prof_begin(ppe_plan_t P, int id) {
  if (!P->prof_on) return -1;
  if (P->prof_used >= kProfMax) {
    ++P->prof_dropped;
    return -1;
  }
  const int r = P->prof_used;
  if ((int)P->prof_ev->size() < 2 * (r + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return -1;
    }
    P->prof_ev->push_back(a);
    P->prof_ev->push_back(b);
    P->prof_name->push_back(id);
  }
  (*P->prof_name)[r] = id;
  cudaEventRecord((*P->prof_ev)[2 * r], P->stream);
  P->prof_used = r + 1;
  return r;
}

void prof_end(ppe_plan_t P, int r) {
  if (r >= 0) cudaEventRecord((*P->prof_ev)[2 * r + 1], P->stream);
}

// Launch with optional per-kernel event bracketing.
#define PPE_LAUNCH(P, ID, expr)             \
  do {                                      \
    const int _r = prof_begin(P, ID);       \
    ppe_status _s = cuda_status(expr);      \
    prof_end(P, _r);                        \
    if (_s != PPE_OK) return _s;            \
  } while (0)

#define PPE_TRY(expr)                      \
  do {                                     \
    ppe_status _s = cuda_status(expr);     \
    if (_s != PPE_OK) return _s;           \
  } while (0)

StencilIn make_in(ppe_plan_t P, const double* u, const double* v, const double* w, const double* S,
                  const double* rho, const double* pn, const double* pnm1, double dt) {
  StencilIn in;
  memset(&in, 0, sizeof(in));
  in.u = u; in.v = v; in.w = w; in.S = S; in.rho = rho; in.pn = pn; in.pnm1 = pnm1;
  in.dt = dt;
  in.inv_dt = dt > 0 ? 1.0 / dt : 0.0;
  in.face_rule = (int)P->opt.face_rule;
  return in;
}

// z forward, y solve, z inverse, x inverse (store or accumulate into p)
template <typename T>
ppe_status solve_tail(ppe_plan_t P, double* p, bool accumulate, bool guarded) {
  const DevScalars* sc = guarded ? P->sc : nullptr;
  cpx<T>* spec = (cpx<T>*)P->spec;
  const double scale = 1.0 / ((double)(P->g.nx / 2) * (double)P->g.nz);
  PPE_LAUNCH(P, K_ZFFT_FWD, launch_zfft<T>(false, P->gd, spec, P->rp_z, (const cpx<T>*)P->tw_z, P->tkx, sc, P->stream));
  PPE_LAUNCH(P, K_YTHOMAS, launch_ythomas<T>(P->gd, spec, (const T*)P->tab, P->line_off, P->line_len, (T)P->a_y, sc, P->stream));
  PPE_LAUNCH(P, K_ZFFT_INV, launch_zfft<T>(true, P->gd, spec, P->rp_z, (const cpx<T>*)P->tw_z, P->tkx, sc, P->stream));
  PPE_LAUNCH(P, accumulate ? K_XINV_ACC : K_XINV, launch_xinv<T>(accumulate, P->gd, spec, p, scale, P->rp_half, (const cpx<T>*)P->tw_x, P->lpb, sc,
                         P->stream));
  return PPE_OK;
}

// The refinement loop of PPE_FP32_REFINE once p holds the first FP32 solve:
// r = f - L p (FP64), delta = L^{-1} r (FP32), p += delta, on the device.
ppe_status refine(ppe_plan_t P, const double* f, double* p) {
  StencilIn in;
  memset(&in, 0, sizeof(in));
  in.f = f;
  in.p = p;
  const int smax = P->opt.max_sweeps;
  cpx<float>* spec = (cpx<float>*)P->spec;
  for (int s = 1; s <= smax; ++s) {
    PPE_LAUNCH(P, K_XFWD_RESID, launch_xfwd<float>(SRC_RESID, true, P->gd, in, P->sc, s, nullptr, spec, P->rp_half,
                               (const cpx<float>*)P->tw_x, P->lpb, P->stream));
    PPE_LAUNCH(P, K_CHECK, launch_refine_check(P->sc, s, smax, P->stream));
    ppe_status st = solve_tail<float>(P, p, true, true);
    if (st != PPE_OK) return st;
  }
  PPE_LAUNCH(P, K_XFWD_RESID, launch_xfwd<float>(SRC_RESID, false, P->gd, in, P->sc, smax + 1, nullptr, spec, P->rp_half,
                             (const cpx<float>*)P->tw_x, P->lpb, P->stream));
  PPE_LAUNCH(P, K_CHECK, launch_refine_check(P->sc, smax + 1, smax, P->stream));
  return PPE_OK;
}

}  // namespace

extern "C" {

int ppe_size_supported(int nx, int ny, int nz) {
  return dim_ok(nx) && dim_ok(ny) && dim_ok(nz) && (nx % 2 == 0) ? 1 : 0;
}

const char* ppe_strerror(ppe_status s) {
  switch (s) {
    case PPE_OK: return "ok";
    case PPE_ERR_INVALID_ARG: return "invalid argument";
    case PPE_ERR_UNSUPPORTED_SIZE: return "unsupported grid size (each dimension 2^a 3^b in [8, 1024], nx even)";
    case PPE_ERR_INCOMPATIBLE_RHS: return "right-hand side incompatible with the Neumann walls";
    case PPE_ERR_OUT_OF_MEMORY: return "device allocation failed";
    case PPE_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
    case PPE_ERR_TIMEOUT: return "device wait timed out";
    case PPE_ERR_CUDA: return "CUDA error";
  }
  return "unknown status";
}

size_t ppe_workspace_bytes(const ppe_grid* g, const ppe_options* opt) {
  if (!g) return 0;
  const bool fp32 = opt && opt->precision == PPE_FP32_REFINE;
  const size_t cb = fp32 ? 8 : 16;
  const size_t n = (size_t)g->nx * g->ny * g->nz;
  const size_t nxh = g->nx / 2 + 1;
  size_t b = cb * nxh * g->ny * g->nz + cb * (g->nx + g->nz) + sizeof(DevScalars);
  if (fp32) b += 8 * n;
  b += (fp32 ? 4 : 8) * nxh * g->nz * (size_t)g->ny + 8 * nxh * g->nz;  // upper bound of the tables
  return b;
}

ppe_status ppe_plan(ppe_plan_t* out, const ppe_grid* g, const ppe_options* opt, void* stream) {
  if (!out || !g) return PPE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(g->lx > 0 && g->ly > 0 && g->lz > 0)) return PPE_ERR_INVALID_ARG;
  if (!ppe_size_supported(g->nx, g->ny, g->nz)) return PPE_ERR_UNSUPPORTED_SIZE;
  ppe_options o;
  o.precision = PPE_FP64;
  o.face_rule = PPE_FACE_ARITHMETIC;
  o.refine_tol = 1e-10;
  o.max_sweeps = 6;
  if (opt) o = *opt;
  if (o.precision != PPE_FP64 && o.precision != PPE_FP32_REFINE) return PPE_ERR_INVALID_ARG;
  if (o.face_rule != PPE_FACE_ARITHMETIC && o.face_rule != PPE_FACE_HARMONIC) return PPE_ERR_INVALID_ARG;
  if (o.max_sweeps < 0 || o.max_sweeps > kMaxSweeps) return PPE_ERR_INVALID_ARG;
  if (o.precision == PPE_FP32_REFINE && !(o.refine_tol >= 0)) return PPE_ERR_INVALID_ARG;

  ppe_plan_t P = new (std::nothrow) ppe_plan_s;
  if (!P) return PPE_ERR_OUT_OF_MEMORY;
  memset(P, 0, sizeof(*P));
  P->prof_ev = new (std::nothrow) std::vector<cudaEvent_t>();
  P->prof_name = new (std::nothrow) std::vector<int>();
  if (!P->prof_ev || !P->prof_name) {
    delete P->prof_ev;
    delete P->prof_name;
    delete P;
    return PPE_ERR_OUT_OF_MEMORY;
  }
  P->g = *g;
  P->opt = o;
  P->stream = (cudaStream_t)stream;
  P->fp32 = o.precision == PPE_FP32_REFINE;
  P->nxh = g->nx / 2 + 1;
  P->gd.nx = g->nx;
  P->gd.ny = g->ny;
  P->gd.nz = g->nz;
  P->gd.idx = g->nx / g->lx;
  P->gd.idy = g->ny / g->ly;
  P->gd.idz = g->nz / g->lz;
  const double dy = g->ly / g->ny;
  P->a_y = 1.0 / (dy * dy);
  P->rp_half = radix_plan(g->nx / 2);
  P->rp_z = radix_plan(g->nz);
  P->lpb = choose_lpb(g->nx);
  P->tkx = choose_tkx(g->nz, P->fp32);
  P->cplx_bytes = P->fp32 ? 8 : 16;

  ppe_status s = PPE_OK;
  const size_t nspec = (size_t)P->nxh * g->ny * g->nz;
  s = alloc_status(cudaMalloc(&P->spec, nspec * P->cplx_bytes));
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->sc, sizeof(DevScalars)));
  if (s == PPE_OK && P->fp32)
    s = alloc_status(cudaMalloc((void**)&P->fbuf, sizeof(double) * (size_t)g->nx * g->ny * g->nz));
  P->workspace = nspec * P->cplx_bytes + sizeof(DevScalars) + (P->fp32 ? 8 * (size_t)g->nx * g->ny * g->nz : 0) +
                 P->cplx_bytes * (g->nx + g->nz);
  if (s == PPE_OK) {
    if (P->fp32) {
      s = make_twiddles<float>(&P->tw_x, g->nx);
      if (s == PPE_OK) s = make_twiddles<float>(&P->tw_z, g->nz);
      if (s == PPE_OK) s = make_thomas<float>(P);
      if (s == PPE_OK) s = cuda_status(set_smem_limits<float>());
    } else {
      s = make_twiddles<double>(&P->tw_x, g->nx);
      if (s == PPE_OK) s = make_twiddles<double>(&P->tw_z, g->nz);
      if (s == PPE_OK) s = make_thomas<double>(P);
      if (s == PPE_OK) s = cuda_status(set_smem_limits<double>());
    }
  }
  if (s == PPE_OK) s = cuda_status(launch_init_scalars(P->sc, -1.0, o.refine_tol, 0, P->stream));
  if (s == PPE_OK) s = cuda_status(cudaStreamSynchronize(P->stream));
  if (s != PPE_OK) {
    ppe_destroy(P);
    return s;
  }
  *out = P;
  return PPE_OK;
}

ppe_status ppe_set_stream(ppe_plan_t P, void* stream) {
  if (!P) return PPE_ERR_INVALID_ARG;
  P->stream = (cudaStream_t)stream;
  return PPE_OK;
}

void ppe_destroy(ppe_plan_t P) {
  if (!P) return;
  cudaFree(P->spec);
  cudaFree(P->tw_x);
  cudaFree(P->tw_z);
  cudaFree(P->tab);
  cudaFree(P->line_off);
  cudaFree(P->line_len);
  cudaFree(P->fbuf);
  cudaFree(P->sc);
  for (int i = 0; i < 12; ++i) cudaFree(P->io[i]);
  if (P->prof_ev)
    for (cudaEvent_t e : *P->prof_ev) cudaEventDestroy(e);
  delete P->prof_ev;
  delete P->prof_name;
  delete P;
}

ppe_status ppe_profile(ppe_plan_t P, int enable) {
  if (!P) return PPE_ERR_INVALID_ARG;
  P->prof_on = enable ? 1 : 0;
  return PPE_OK;
}

int ppe_profile_read(ppe_plan_t P, ppe_kernel_time* out, int max_entries) {
  if (!P || !out || max_entries <= 0) return -1;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return -1;
  int launches[K_COUNT] = {0};
  double ms[K_COUNT] = {0};
  for (int r = 0; r < P->prof_used; ++r) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, (*P->prof_ev)[2 * r], (*P->prof_ev)[2 * r + 1]) != cudaSuccess) continue;
    const int id = (*P->prof_name)[r];
    launches[id] += 1;
    ms[id] += t;
  }
  int n = 0;
  for (int id = 0; id < K_COUNT && n < max_entries; ++id) {
    if (!launches[id]) continue;
    memset(&out[n], 0, sizeof(out[n]));
    strncpy(out[n].name, kKernelNames[id], sizeof(out[n].name) - 1);
    out[n].launches = launches[id];
    out[n].total_ms = ms[id];
    ++n;
  }
  P->prof_used = 0;
  P->prof_dropped = 0;
  return n;
}

ppe_status ppe_rhs(ppe_plan_t P, const double* u, const double* v, const double* w, const double* S,
                   const double* rho, const double* p_n, const double* p_nm1, double rho0, double dt, double* f) {
  if (!P || !u || !v || !w || !S || !rho || !p_n || !p_nm1 || !f || !(dt > 0)) return PPE_ERR_INVALID_ARG;
  StencilIn in = make_in(P, u, v, w, S, rho, p_n, p_nm1, dt);
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  PPE_LAUNCH(P, K_INIT, launch_init_scalars(P->sc, rho0, P->opt.refine_tol, 0, P->stream));
  if (!(rho0 > 0)) PPE_LAUNCH(P, K_RHO_MIN, launch_rho_min(rho, n, P->sc, P->stream));
  if (P->fp32)
    PPE_LAUNCH(P, K_XFWD_RHS, launch_xfwd<float>(SRC_RHS, false, P->gd, in, P->sc, 0, f, nullptr, P->rp_half, nullptr, P->lpb,
                               P->stream));
  else
    PPE_LAUNCH(P, K_XFWD_RHS, launch_xfwd<double>(SRC_RHS, false, P->gd, in, P->sc, 0, f, nullptr, P->rp_half, nullptr, P->lpb,
                                P->stream));
  return PPE_OK;
}

ppe_status ppe_solve(ppe_plan_t P, const double* f, double* p) {
  if (!P || !f || !p) return PPE_ERR_INVALID_ARG;
  StencilIn in;
  memset(&in, 0, sizeof(in));
  in.f = f;
  PPE_LAUNCH(P, K_INIT, launch_init_scalars(P->sc, -1.0, P->opt.refine_tol, 1, P->stream));
  if (P->fp32) {
    PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<float>(SRC_F, true, P->gd, in, P->sc, 0, nullptr, (cpx<float>*)P->spec, P->rp_half,
                               (const cpx<float>*)P->tw_x, P->lpb, P->stream));
    ppe_status s = solve_tail<float>(P, p, false, false);
    if (s != PPE_OK) return s;
    return refine(P, f, p);
  }
  PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<double>(SRC_F, true, P->gd, in, P->sc, 0, nullptr, (cpx<double>*)P->spec, P->rp_half,
                              (const cpx<double>*)P->tw_x, P->lpb, P->stream));
  return solve_tail<double>(P, p, false, false);
}

ppe_status ppe_correct(ppe_plan_t P, const double* u, const double* v, const double* w, const double* rho,
                       const double* p, const double* p_n, const double* p_nm1, double rho0, double dt,
                       double* u_out, double* v_out, double* w_out) {
  if (!P || !u || !v || !w || !rho || !p || !p_n || !p_nm1 || !u_out || !v_out || !w_out || !(dt > 0))
    return PPE_ERR_INVALID_ARG;
  StencilIn in = make_in(P, u, v, w, nullptr, rho, p_n, p_nm1, dt);
  in.p = p;
  if (rho0 > 0) PPE_TRY(launch_set_rho0(P->sc, rho0, P->stream));
  PPE_LAUNCH(P, K_CORRECT, launch_correct(P->gd, in, P->sc, u_out, v_out, w_out, P->stream));
  return PPE_OK;
}

ppe_status ppe_project(ppe_plan_t P, const ppe_fields* F) {
  if (!P || !F || !F->u || !F->v || !F->w || !F->S || !F->rho || !F->p_n || !F->p_nm1 || !F->p || !F->u_out ||
      !F->v_out || !F->w_out || !(F->dt > 0))
    return PPE_ERR_INVALID_ARG;
  StencilIn in = make_in(P, F->u, F->v, F->w, F->S, F->rho, F->p_n, F->p_nm1, F->dt);
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  PPE_LAUNCH(P, K_INIT, launch_init_scalars(P->sc, F->rho0, P->opt.refine_tol, 0, P->stream));
  if (!(F->rho0 > 0)) PPE_LAUNCH(P, K_RHO_MIN, launch_rho_min(F->rho, n, P->sc, P->stream));
  ppe_status s;
  if (P->fp32) {
    double* f = F->f ? F->f : P->fbuf;
    PPE_LAUNCH(P, K_XFWD_RHS, launch_xfwd<float>(SRC_RHS, true, P->gd, in, P->sc, 0, f, (cpx<float>*)P->spec, P->rp_half,
                               (const cpx<float>*)P->tw_x, P->lpb, P->stream));
    if ((s = solve_tail<float>(P, F->p, false, false)) != PPE_OK) return s;
    if ((s = refine(P, f, F->p)) != PPE_OK) return s;
  } else {
    PPE_LAUNCH(P, K_XFWD_RHS, launch_xfwd<double>(SRC_RHS, true, P->gd, in, P->sc, 0, F->f, (cpx<double>*)P->spec, P->rp_half,
                                (const cpx<double>*)P->tw_x, P->lpb, P->stream));
    if ((s = solve_tail<double>(P, F->p, false, false)) != PPE_OK) return s;
  }
  in.p = F->p;
  PPE_LAUNCH(P, K_CORRECT, launch_correct(P->gd, in, P->sc, F->u_out, F->v_out, F->w_out, P->stream));
  return PPE_OK;
}

ppe_status ppe_project_host(ppe_plan_t P, const ppe_fields* H) {
  if (!P || !H || !H->u || !H->v || !H->w || !H->S || !H->rho || !H->p_n || !H->p_nm1 || !H->p || !H->u_out ||
      !H->v_out || !H->w_out || !(H->dt > 0))
    return PPE_ERR_INVALID_ARG;
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  const size_t nv = (size_t)P->g.nx * (P->g.ny + 1) * P->g.nz;
  // staging: 0 u, 1 v, 2 w, 3 S, 4 rho, 5 p_n, 6 p_nm1, 7 p, 8 f
  const size_t sizes[9] = {n, nv, n, n, n, n, n, n, n};
  const int nbuf = H->f ? 9 : 8;
  for (int i = 0; i < nbuf; ++i)
    if (!P->io[i]) {
      ppe_status s = alloc_status(cudaMalloc((void**)&P->io[i], sizes[i] * sizeof(double)));
      if (s != PPE_OK) return s;
    }
  const double* src[7] = {H->u, H->v, H->w, H->S, H->rho, H->p_n, H->p_nm1};
  for (int i = 0; i < 7; ++i)
    PPE_TRY(cudaMemcpyAsync(P->io[i], src[i], sizes[i] * sizeof(double), cudaMemcpyHostToDevice, P->stream));
  ppe_fields D;
  D.u = P->io[0]; D.v = P->io[1]; D.w = P->io[2]; D.S = P->io[3]; D.rho = P->io[4];
  D.p_n = P->io[5]; D.p_nm1 = P->io[6];
  D.rho0 = H->rho0;
  D.dt = H->dt;
  D.p = P->io[7];
  D.u_out = P->io[0]; D.v_out = P->io[1]; D.w_out = P->io[2];  // in place
  D.f = H->f ? P->io[8] : nullptr;
  ppe_status s = ppe_project(P, &D);
  if (s != PPE_OK) return s;
  PPE_TRY(cudaMemcpyAsync(H->p, D.p, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaMemcpyAsync(H->u_out, D.u_out, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaMemcpyAsync(H->v_out, D.v_out, nv * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaMemcpyAsync(H->w_out, D.w_out, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  if (H->f) PPE_TRY(cudaMemcpyAsync(H->f, D.f, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaStreamSynchronize(P->stream));
  return PPE_OK;
}

ppe_status ppe_get_info(ppe_plan_t P, ppe_info* info) {
  if (!P || !info) return PPE_ERR_INVALID_ARG;
  DevScalars h;
  PPE_TRY(cudaMemcpyAsync(&h, P->sc, sizeof(h), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaStreamSynchronize(P->stream));
  const double fmax = h.fmax_bits ? __builtin_bit_cast(double, h.fmax_bits) : 0.0;
  info->f_max = fmax;
  info->rho0 = __builtin_bit_cast(double, h.rho0_bits);
  if (P->fp32) {
    info->sweeps = h.sweeps;
    if (h.last_slot >= 0 && fmax > 0)
      info->rel_residual = __builtin_bit_cast(double, h.rmax_bits[h.last_slot]) / fmax;
    else
      info->rel_residual = -1.0;
    if (h.last_slot >= 0 && !h.done) return PPE_ERR_NOT_CONVERGED;
  } else {
    info->sweeps = 0;
    info->rel_residual = -1.0;
  }
  return PPE_OK;
}

}  // extern "C"
