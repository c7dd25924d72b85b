// Host side of libppe: plans, tables and the C entry points declared in
// include/ppe.h (split pressure-gradient projection, Sec. 5.4 of the paper,
// Eqs. (32)-(34)).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost a pointer test when no tool is attached

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
  bool pairs;         // PPE_FP64 with walls: transforms and y solve in double-float pairs (dd)
  size_t cplx_bytes;
  void* spec;         // cpx<T>[nz][ny][nxh]
  void* tw_x;         // cpx<T>[nx]: exp(-2 pi i t/nx)
  void* tw_z;         // cpx<T>[nz]
  void* tab;          // T: elimination multipliers (FP64 form)
  RadixPlan rp_y;     // ny (FP32 form: DCT along y)
  void* tw_y;         // cpx<T>[ny]: exp(-2 pi i t/ny)
  void* wq_y;         // cpx<T>[ny]: exp(-i pi k/(2 ny))
  void* lam;          // T[nxh + ny + nz]: eigenvalue parts lam_x, lam_y, lam_z
  int tky;            // kx columns per CTA of the y DCT pass
  int* line_off;
  int* line_len;
  double a_y;         // 1/dy^2
  int tj, kc;         // right-hand-side kernel: lines per tile, planes per chunk
  df* fdf;            // FP32_REFINE: right-hand side as pairs, kept for the residual
  df* pdf;            // FP32_REFINE: pressure as pairs during the refinement
  float* p32;         // FP32_REFINE, register-staged x passes, (nx/2) nz a power of two, max_sweeps >= 1:
                      // ppe_project's first-solve p in FP32 (a pair with a zero low part), read by the
                      // first sweep's residual and accumulation
  df* upre;           // explicitly split velocity u_pre on x faces (ppe_project)
  df* vpre;           //   ... on y faces
  df* wpre;           //   ... on z faces
  double2* rhs_part;  // per-CTA partial sums (3 ny nz entries: right-hand side, forward and inverse x transforms)
  DevScalars* sc;
  // spectral schedule (ppe_tuning.spectral): FUSED (k_zyz.cu) where zyz_ok, PENCIL
  // (k_pencil.cu) where pencil_ok; both keep the spectrum in the plane layout
  // (gd.spec_planes), mapped by tmap (a fused pass's tile) and tmap_z (a z tile)
  bool zyz_ok;
  bool pencil_ok;
  int sched;
  // y step of the LEGACY schedule (ppe_tuning.y_solve): PPE_Y_TRIDIAGONAL where
  // yscan_ok (FP32_REFINE, walls, ny <= 512: Thomas tables built)
  bool yscan_ok;
  int y_solve;
  alignas(64) CUtensorMap tmap;
  alignas(64) CUtensorMap tmap_z;
  // refinement loops as CUDA graphs with a WHILE conditional node (FP32_REFINE):
  // ppe_solve's and ppe_project's (the latter ends with the fused correction)
  cudaGraphExec_t refine_exec;
  cudaGraphExec_t project_exec;
  // unsplit projection (ppe_project_unsplit; allocated on first use): face
  // coefficients, CG vectors, partial sums, the iteration graph
  df* vc[8];          // ax, ay, az, x, r, p, Kp, zs
  double2* pcg_part;
  cudaGraphExec_t pcg_exec;
  // ppe_project_host staging (allocated on first use)
  double* io[12];
  // ppe_project_host_async: two staging sets used in turn, copy-in and
  // copy-out streams, per-set events, the scalars of each set's projection
  // (pinned host memory), and what the pipeline has retired so far
  double* aio[2][9];
  cudaStream_t acin, acout;
  cudaEvent_t aev_in[2], aev_done[2], aev_out[2];
  DevScalars* ahsc;   // [2], pinned
  int aset;           // set of the next call
  int abusy[2];       // set holds a call not yet retired
  ppe_status astatus; // first non-OK status of the calls retired since the last ppe_host_wait
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

// Radix sequence: radix 16 while it divides (up to maxr), one 8, 4s, one 2,
// then 3s -- the fewest shared-memory passes for 2^a 3^b.
RadixPlan radix_plan(int n, int maxr) {
  RadixPlan rp;
  memset(&rp, 0, sizeof(rp));
  rp.n = n;
  int m = n;
  while (maxr >= 16 && m % 16 == 0) { rp.r[rp.nst++] = 16; m /= 16; }
  if (maxr >= 8 && m % 8 == 0) { rp.r[rp.nst++] = 8; m /= 8; }
  while (m % 4 == 0) { rp.r[rp.nst++] = 4; m /= 4; }
  if (m % 2 == 0) { rp.r[rp.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { rp.r[rp.nst++] = 3; m /= 3; }
  int ns = 1;
  for (int s = 0; s < rp.nst; ++s) {
    rp.ns[s] = make_fastdiv((uint32_t)ns);
    ns *= rp.r[s];
  }
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
      // walls: the kx = kz = 0 line is singular and pinned by the kernel; an open
      // top (ghost -p above the last cell) makes the last diagonal -3a + lam
      // and every line regular
      const bool open = P->gd.top_open != 0;
      const bool zero = !open && kx == 0 && kz == 0;
      m[0] = zero ? 0.0 : 1.0 / (-a + lam);
      for (int j = 1; j < ny - 1; ++j) m[j] = 1.0 / ((-2.0 * a + lam) - a * (a * m[j - 1]));
      m[ny - 1] = 1.0 / (((open ? -3.0 : -1.0) * a + lam) - a * (a * m[ny - 2]));
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

// lines per CTA of the x passes: the largest power of two <= 2048/nx, in [1, 64]
// Eigenvalue parts of the 7-point operator (FP64 on the host, rounded to T):
// lam_x(kx) = -(4/dx^2) sin^2(pi kx/nx), lam_y(ky) = -(4/dy^2) sin^2(pi ky/(2 ny)),
// lam_z(kz) = -(4/dz^2) sin^2(pi kz/nz), and the quarter-wave factors of the DCT.
template <typename T>
ppe_status make_dct_tables(ppe_plan_t P) {
  const int nx = P->g.nx, ny = P->g.ny, nz = P->g.nz, nxh = P->nxh;
  const double dx = P->g.lx / nx, dy = P->g.ly / ny, dz = P->g.lz / nz;
  std::vector<T> lam(nxh + ny + nz);
  for (int k = 0; k < nxh; ++k) {
    const double s = sin_pi_frac(k, nx);
    lam[k] = (T)(-(4.0 / (dx * dx)) * s * s);
  }
  for (int k = 0; k < ny; ++k) {
    const double s = sin_pi_frac(k, 2 * ny);
    lam[nxh + k] = (T)(-(4.0 / (dy * dy)) * s * s);
  }
  for (int k = 0; k < nz; ++k) {
    const double s = sin_pi_frac(k, nz);
    lam[nxh + ny + k] = (T)(-(4.0 / (dz * dz)) * s * s);
  }
  std::vector<cpx<T>> wq(ny);
  for (int k = 0; k < ny; ++k) {
    double re, im;
    cis_neg(k, 4 * ny, &re, &im);  // exp(-2 pi i k/(4 ny)) = exp(-i pi k/(2 ny))
    wq[k].x = (T)re;
    wq[k].y = (T)im;
  }
  ppe_status s;
  if ((s = upload(&P->lam, lam)) != PPE_OK) return s;
  if ((s = upload(&P->wq_y, wq)) != PPE_OK) return s;
  if ((s = make_twiddles<T>(&P->tw_y, ny)) != PPE_OK) return s;
  P->workspace += lam.size() * sizeof(T) + 2 * sizeof(cpx<T>) * ny;
  return PPE_OK;
}

int choose_lpb(int nx) {
  int l = 1;
  while (2 * l <= 4096 / nx && 2 * l <= 64) l *= 2;
  return l;
}

// kx columns per CTA of the z and y passes: 16 for the FP32 z pass (128-byte
// rows), 8 otherwise (64-byte FP32 / 128-byte FP64 rows) -- measured best at
// 256^3 on a GB300 -- fewer when the tile would not fit
int choose_tkx(int nz, bool fp32, bool zpass) {
  const size_t cb = fp32 ? 8 : 16;
  int t = (fp32 && zpass) ? 16 : 8;
  while (t > 2 && cb * (2 * (size_t)t * nz + nz) > 160 * 1024) t /= 2;
  return t;
}

ppe_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PPE_OK : PPE_ERR_CUDA; }

// cuTensorMapEncodeTiled from the driver, looked up through the runtime (no
// link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
      cudaGetLastError();
      return nullptr;
    }
    fn = (EncodeTiledFn)f;
  }
  return fn;
}

// The spectrum in the plane layout as a 2-D tensor of 8-byte elements (one
// complex FP32 value each): x = j (ny), y = kx nz + kz; a box is zyz_cols(ny, nz)
// columns of j by nz rows of kz, i.e. one CTA's tile of one kx plane.  Row
// pitch ny * 8 bytes (a multiple of 16 for every supported ny).
bool make_spec_tmap(ppe_plan_t P, CUtensorMap* map, int box_cols) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const int ny = P->g.ny, nz = P->g.nz, nxh = P->nxh;
  const cuuint64_t dims[2] = {(cuuint64_t)ny, (cuuint64_t)nz * (cuuint64_t)nxh};
  const cuuint64_t strides[1] = {(cuuint64_t)ny * 8u};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)nz};
  const cuuint32_t es[2] = {1u, 1u};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, P->spec, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool sched_ok(ppe_plan_t P, int s) {
  return s == PPE_SPECTRAL_LEGACY || (s == PPE_SPECTRAL_FUSED && P->zyz_ok) ||
         (s == PPE_SPECTRAL_PENCIL && P->pencil_ok);
}

void set_sched(ppe_plan_t P, int s) {
  P->sched = sched_ok(P, s) ? s : PPE_SPECTRAL_LEGACY;
  P->gd.spec_planes = P->sched != PPE_SPECTRAL_LEGACY ? 1 : 0;
}

// Kernel names reported by ppe_profile_read.
enum KernelId { K_INIT, K_RHO_MIN, K_RHS, K_XFWD_F, K_XFWD_RESID, K_ZFFT_FWD, K_YTHOMAS, K_ZFFT_INV,
                K_XINV, K_XINV_ACC, K_CORRECT, K_CHECK, K_DF_TO_D, K_VC_SETUP, K_VC_APPLY, K_VC_UPDATE,
                K_VC_DOTS, K_VC_PUPDATE, K_VC_SCALAR, K_VC_CORRECT, K_DIV_S, K_CONST, K_ZYZ, K_COUNT };
const char* const kKernelNames[K_COUNT] = {"k_init_scalars", "k_rho_min", "k_rhs_march", "k_xfwd_f",
                                           "k_xfwd_resid", "k_zfft_fwd", "k_ysolve", "k_zfft_inv",
                                           "k_xinv", "k_xinv_accum", "k_correct", "k_refine_check",
                                           "k_df_to_d", "k_vc_setup", "k_vc_apply", "k_vc_update",
                                           "k_vc_dots", "k_vc_pupdate", "k_vc_scalars", "k_vc_correct",
                                           "k_div_constraint", "k_make_const", "k_zyz"};
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
// Every launch of the path: an NVTX range named after the kernel (for
// timeline tools), the optional per-kernel event timing, the status check.
#define PPE_LAUNCH(P, ID, expr)             \
  do {                                      \
    nvtxRangePushA(kKernelNames[ID]);       \
    const int _r = prof_begin(P, ID);       \
    ppe_status _s = cuda_status(expr);      \
    prof_end(P, _r);                        \
    nvtxRangePop();                         \
    if (_s != PPE_OK) return _s;            \
  } while (0)

// NVTX range over one call of the C ABI
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

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

// z forward, y solve, z inverse, x inverse (mode XI_F64: p64 = x; XI_DF:
// pdf = x; XI_DF_ACC: pdf += x).  psum: the x inverse also sums the p it writes,
// and the next solve's zero mode takes minus that sum (the refinement keeps p
// zero-mean); off where the solve is a preconditioner, not a pressure.
template <typename T>
ppe_status solve_tail(ppe_plan_t P, int mode, double* p64, df* pdf, bool guarded, bool psum = true,
                      float* p32 = nullptr) {
  DevScalars* psc = (psum && mode != XI_F64) ? P->sc : nullptr;
  const DevScalars* sc = guarded ? P->sc : nullptr;
  cpx<T>* spec = (cpx<T>*)P->spec;
  const double scale = 1.0 / ((double)(P->g.nx / 2) * (double)P->g.nz);
  // the first pass after an x transform of f also totals the partial sums (finish_sums)
  DevScalars* fin = guarded ? nullptr : P->sc;
  if (P->sched != PPE_SPECTRAL_LEGACY) {
    const float* lam = (const float*)P->lam;
    const cpx<float>* twz = (const cpx<float>*)P->tw_z;
    const cpx<float>* twy = (const cpx<float>*)P->tw_y;
    const cpx<float>* wqy = (const cpx<float>*)P->wq_y;
    const float *lx = lam, *ly = lam + P->nxh, *lz = lam + P->nxh + P->g.ny;
    if (P->sched == PPE_SPECTRAL_FUSED) {
      PPE_LAUNCH(P, K_ZYZ, launch_zyz(P->gd, P->tmap, twz, twy, wqy, lx, ly, lz, P->sc, fin, P->stream));
    } else {
      PPE_LAUNCH(P, K_ZFFT_FWD, launch_zfft_tma(false, P->gd, P->tmap_z, twz, P->sc, fin, P->stream));
      PPE_LAUNCH(P, K_YTHOMAS, launch_ydct_tma(P->gd, (cpx<float>*)P->spec, twy, wqy, lx, ly, lz, P->sc,
                                               P->stream));
      PPE_LAUNCH(P, K_ZFFT_INV, launch_zfft_tma(true, P->gd, P->tmap_z, twz, P->sc, nullptr, P->stream));
    }
    PPE_LAUNCH(P, mode == XI_DF_ACC ? K_XINV_ACC : K_XINV,
               launch_xinv<T>(mode, P->gd, spec, p64, pdf, scale, P->rp_half, (const cpx<T>*)P->tw_x, P->lpb, sc,
                              psc, P->stream, p32));
    return PPE_OK;
  }
  PPE_LAUNCH(P, K_ZFFT_FWD,
             launch_zfft<T>(false, P->gd, spec, P->rp_z, (const cpx<T>*)P->tw_z, P->tkx, sc, fin, P->stream));
  if (P->y_solve == PPE_Y_TRIDIAGONAL) {  // (FP32, walls) the Thomas elimination in scan form
    PPE_LAUNCH(P, K_YTHOMAS, launch_ythomas_scan(P->gd, (cpx<float>*)spec, (const float*)P->tab, P->line_off,
                                                 P->line_len, (float)P->a_y, P->sc, P->stream));
  } else if ((P->fp32 || P->pairs) && !P->gd.top_open) {  // DCT-II/III for walls; the open top: tridiagonal solve
    const T* lam = (const T*)P->lam;
    PPE_LAUNCH(P, K_YTHOMAS, launch_ydct<T>(P->gd, spec, P->rp_y, (const cpx<T>*)P->tw_y, (const cpx<T>*)P->wq_y,
                                            lam, lam + P->nxh, lam + P->nxh + P->g.ny, P->tky, P->sc, P->stream));
  } else {
    PPE_LAUNCH(P, K_YTHOMAS, launch_ythomas<T>(P->gd, spec, (const T*)P->tab, P->line_off, P->line_len, (T)P->a_y,
                                               sc, P->stream));
  }
  PPE_LAUNCH(P, K_ZFFT_INV,
             launch_zfft<T>(true, P->gd, spec, P->rp_z, (const cpx<T>*)P->tw_z, P->tkx, sc, nullptr, P->stream));
  PPE_LAUNCH(P, mode == XI_DF_ACC ? K_XINV_ACC : K_XINV,
             launch_xinv<T>(mode, P->gd, spec, p64, pdf, scale, P->rp_half, (const cpx<T>*)P->tw_x, P->lpb, sc,
                            psc, P->stream, p32));
  return PPE_OK;
}

// Runs f(T{}) with T the element type of a PPE_FP64 plan's spectral passes:
// double-float pairs with walls, native FP64 with an outflow top.
template <typename F>
ppe_status with_fp64_type(ppe_plan_t P, F&& f) {
  if (P->pairs) return f(dd(0));
  return f(0.0);
}

// Refinement sequences of PPE_FP32_REFINE (after the first FP32 solve left p
// in pdf).  Residuals go into slot sc->iter (see k_refine_check).
//   REF_SOLVE   (ppe_solve):   probe; WHILE(cont) { p += L^{-1} r; probe }
//               probe = residual r = f - L p with its x transform, test.
//   REF_PROJECT (ppe_project): WHILE(cont) { r = f - L p + x transform;
//               p += L^{-1} r; Eq. (33) correction fused with the residual of
//               the new p; test }  -- at least one correction, and the test
//               after the last correction needs no separate residual pass.
enum RefMode { REF_SOLVE = 0, REF_PROJECT = 1 };

// p0f: the first solve's p in FP32 (read at the first sweep), or NULL
ppe_status resid_fwd(ppe_plan_t P, const float* p0f) {
  StencilIn in;
  memset(&in, 0, sizeof(in));
  in.p0f = p0f;
  PPE_LAUNCH(P, K_XFWD_RESID, launch_xfwd<float>(SRC_RESID, true, P->gd, in, P->sc, -1, P->fdf, P->pdf,
                                                 (cpx<float>*)P->spec, P->rp_half, (const cpx<float>*)P->tw_x,
                                                 P->lpb, P->stream));
  return PPE_OK;
}

ppe_status refine_probe(ppe_plan_t P, cudaGraphConditionalHandle h, int use_handle) {
  ppe_status s = resid_fwd(P, nullptr);
  if (s != PPE_OK) return s;
  PPE_LAUNCH(P, K_CHECK, launch_refine_check(P->sc, P->opt.max_sweeps, 0, h, use_handle, P->stream));
  return PPE_OK;
}

ppe_status refine_body(ppe_plan_t P, int mode, cudaGraphConditionalHandle h, int use_handle) {
  ppe_status s;
  if (mode == REF_SOLVE) {
    if ((s = solve_tail<float>(P, XI_DF_ACC, nullptr, P->pdf, false)) != PPE_OK) return s;
    return refine_probe(P, h, use_handle);
  }
  if ((s = resid_fwd(P, P->p32)) != PPE_OK) return s;
  if ((s = solve_tail<float>(P, XI_DF_ACC, nullptr, P->pdf, false, true, P->p32)) != PPE_OK) return s;
  PPE_LAUNCH(P, K_CORRECT, launch_correct_check(P->gd, P->upre, P->vpre, P->wpre, P->pdf, P->fdf, P->sc, P->stream));
  PPE_LAUNCH(P, K_CHECK, launch_refine_check(P->sc, P->opt.max_sweeps, 1, h, use_handle, P->stream));
  return PPE_OK;
}

// Appends a refinement sequence to the graph that P->stream is capturing:
// [probe]; WHILE(cond) { body }, the condition set on the device by the test
// kernel.  Used to build the per-plan refinement graphs and, when a caller
// captures ppe_project (e.g. ppe_batch_create), inline in the caller's graph.
ppe_status capture_refine(ppe_plan_t P, int mode) {
  const int saved_prof = P->prof_on;
  P->prof_on = 0;
  cudaStream_t cs = P->stream;
  cudaStream_t bs = nullptr;
  ppe_status st = PPE_OK;
  auto done = [&](ppe_status s) {
    P->stream = cs;
    P->prof_on = saved_prof;
    if (bs) cudaStreamDestroy(bs);
    if (s != PPE_OK) cudaGetLastError();
    return s;
  };
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess ||
      cst != cudaStreamCaptureStatusActive)
    return done(PPE_ERR_CUDA);
  cudaGraphConditionalHandle h;
  // REF_PROJECT runs its body at least once: the condition starts at 1
  if (cudaGraphConditionalHandleCreate(&h, cg, mode == REF_PROJECT ? 1u : 0u, cudaGraphCondAssignDefault) !=
      cudaSuccess)
    return done(PPE_ERR_CUDA);
  if (mode == REF_SOLVE) {
    if ((st = refine_probe(P, h, 1)) != PPE_OK) return done(st);
    if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess)
      return done(PPE_ERR_CUDA);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cond = nullptr;
  if (cudaGraphAddNode(&cond, cg, deps, nullptr, ndeps, &cp) != cudaSuccess) return done(PPE_ERR_CUDA);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return done(PPE_ERR_CUDA);
  // the body is captured from a second stream into the conditional's graph
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return done(PPE_ERR_CUDA);
  if (cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return done(PPE_ERR_CUDA);
  P->stream = bs;
  st = refine_body(P, mode, h, 1);
  P->stream = cs;
  cudaGraph_t outb = nullptr;
  if (cudaStreamEndCapture(bs, &outb) != cudaSuccess && st == PPE_OK) st = PPE_ERR_CUDA;
  return done(st);
}

// Builds a refinement graph once per plan (it touches plan-owned buffers and
// the device scalar block only).
ppe_status build_refine_graph(ppe_plan_t P, int mode, cudaGraphExec_t* exec) {
  cudaStream_t saved = P->stream;
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  auto fail = [&](ppe_status s) {
    P->stream = saved;
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    cudaGetLastError();
    return s;
  };
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(PPE_ERR_CUDA);
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return fail(PPE_ERR_CUDA);
  if (cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(PPE_ERR_CUDA);
  P->stream = cs;
  ppe_status st = capture_refine(P, mode);
  P->stream = saved;
  cudaGraph_t outg = nullptr;
  if (cudaStreamEndCapture(cs, &outg) != cudaSuccess) {
    // an invalidated capture leaves the graph to the runtime: it is not
    // destroyed here (a second destroy of a released graph crashes the process)
    g = nullptr;
    if (st == PPE_OK) st = PPE_ERR_CUDA;
  }
  if (st != PPE_OK) return fail(st);
  if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) return fail(PPE_ERR_CUDA);
  cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return PPE_OK;
}

ppe_status build_refine_graphs(ppe_plan_t P) {
  if (P->refine_exec) cudaGraphExecDestroy(P->refine_exec);
  if (P->project_exec) cudaGraphExecDestroy(P->project_exec);
  P->refine_exec = nullptr;
  P->project_exec = nullptr;
  ppe_status s = build_refine_graph(P, REF_SOLVE, &P->refine_exec);
  if (s == PPE_OK) s = build_refine_graph(P, REF_PROJECT, &P->project_exec);
  return s;
}

// ---- unsplit projection (Eqs. (29)-(30)) by preconditioned conjugate gradients ----
enum { VC_AX, VC_AY, VC_AZ, VC_X, VC_R, VC_P, VC_KP, VC_ZS };

ppe_status ensure_vc(ppe_plan_t P) {
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  for (int i = 0; i < 8; ++i)
    if (!P->vc[i]) {
      ppe_status s = alloc_status(cudaMalloc((void**)&P->vc[i], sizeof(df) * n));
      if (s != PPE_OK) return s;
    }
  if (!P->pcg_part) return alloc_status(cudaMalloc((void**)&P->pcg_part, sizeof(double2) * vc_grid(n)));
  return PPE_OK;
}

VcConst make_vc_const(const ppe_grid& g, double dt) {
  const double hx = g.lx / g.nx, hy = g.ly / g.ny, hz = g.lz / g.nz;
  VcConst C;
  C.ix2 = d2df(1.0 / (hx * hx));
  C.iy2 = d2df(1.0 / (hy * hy));
  C.iz2 = d2df(1.0 / (hz * hz));
  C.idx = d2df(1.0 / hx);
  C.idy = d2df(1.0 / hy);
  C.idz = d2df(1.0 / hz);
  C.idt = d2df(1.0 / dt);
  C.dthx = d2df(dt * hx);
  C.dthy = d2df(dt * hy);
  C.dthz = d2df(dt * hz);
  return C;
}

// zs = L^{-1} r by the plan's FFT solve (the preconditioner is z = -zs)
ppe_status vc_precond(ppe_plan_t P) {
  StencilIn in;
  memset(&in, 0, sizeof(in));
  df* r = P->vc[VC_R];
  df* zs = P->vc[VC_ZS];
  if (P->fp32) {
    PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<float>(SRC_FDF, true, P->gd, in, P->sc, 0, r, nullptr, (cpx<float>*)P->spec,
                                               P->rp_half, (const cpx<float>*)P->tw_x, P->lpb, P->stream));
    return solve_tail<float>(P, XI_DF, nullptr, zs, false, false);
  }
  return with_fp64_type(P, [&](auto tag) -> ppe_status {
    using T = decltype(tag);
    PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<T>(SRC_FDF, true, P->gd, in, P->sc, 0, r, nullptr, (cpx<T>*)P->spec,
                                           P->rp_half, (const cpx<T>*)P->tw_x, P->lpb, P->stream));
    return solve_tail<T>(P, XI_DF, nullptr, zs, false, false);
  });
}

// One iteration: Kp, alpha, x and r, z = M^{-1} r, beta and the test, p.
ppe_status vc_iteration(ppe_plan_t P, cudaGraphConditionalHandle h, int use_handle) {
  df** V = P->vc;
  PPE_LAUNCH(P, K_VC_APPLY, launch_vc_apply(P->gd, V[VC_P], V[VC_AX], V[VC_AY], V[VC_AZ], V[VC_KP], P->pcg_part,
                                            P->stream));
  PPE_LAUNCH(P, K_VC_SCALAR, launch_vc_alpha(P->gd, P->sc, P->pcg_part, P->stream));
  PPE_LAUNCH(P, K_VC_UPDATE, launch_vc_update(P->gd, V[VC_X], V[VC_R], V[VC_P], V[VC_KP], P->sc, P->stream));
  ppe_status s = vc_precond(P);
  if (s != PPE_OK) return s;
  PPE_LAUNCH(P, K_VC_DOTS, launch_vc_dots(P->gd, V[VC_R], V[VC_ZS], V[VC_KP], P->pcg_part, P->stream));
  PPE_LAUNCH(P, K_VC_SCALAR, launch_vc_beta(P->gd, P->sc, P->pcg_part, 0, h, use_handle, P->stream));
  PPE_LAUNCH(P, K_VC_PUPDATE, launch_vc_pupdate(P->gd, V[VC_P], V[VC_ZS], P->sc, P->stream));
  return PPE_OK;
}

// The iteration loop as a graph: WHILE(cond) { iteration }, the condition
// (default 1) set on the device by the beta kernel.  Built once per plan; it
// touches plan-owned buffers and the device scalar block only.
ppe_status build_pcg_graph(ppe_plan_t P) {
  const int saved_prof = P->prof_on;
  cudaStream_t saved = P->stream;
  cudaStream_t cs = nullptr, bs = nullptr;
  cudaGraph_t g = nullptr;
  auto fail = [&](ppe_status s) {
    P->stream = saved;
    P->prof_on = saved_prof;
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    if (bs) cudaStreamDestroy(bs);
    cudaGetLastError();
    return s;
  };
  P->prof_on = 0;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return fail(PPE_ERR_CUDA);
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(PPE_ERR_CUDA);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cond = nullptr;
  if (cudaGraphAddNode(&cond, g, nullptr, nullptr, 0, &cp) != cudaSuccess) return fail(PPE_ERR_CUDA);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return fail(PPE_ERR_CUDA);
  if (cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(PPE_ERR_CUDA);
  P->stream = bs;
  ppe_status st = vc_iteration(P, h, 1);
  P->stream = saved;
  cudaGraph_t outb = nullptr;
  if (cudaStreamEndCapture(bs, &outb) != cudaSuccess && st == PPE_OK) st = PPE_ERR_CUDA;
  if (st != PPE_OK) return fail(st);
  if (cudaGraphInstantiate(&P->pcg_exec, g, 0) != cudaSuccess) return fail(PPE_ERR_CUDA);
  cudaGraphDestroy(g);
  cudaStreamDestroy(bs);
  P->prof_on = saved_prof;
  return PPE_OK;
}

// Runs a refinement sequence.  Normally one graph launch (the loop runs on the
// device); while per-kernel profiling is on, the same kernels are launched from
// the host, which reads the test result after each check.
ppe_status refine(ppe_plan_t P, int mode) {
  if (mode == REF_PROJECT && P->opt.max_sweeps == 0) {
    cudaGraphConditionalHandle none = 0;
    PPE_LAUNCH(P, K_CORRECT, launch_correct_check(P->gd, P->upre, P->vpre, P->wpre, P->pdf, P->fdf, P->sc,
                                                  P->stream));
    PPE_LAUNCH(P, K_CHECK, launch_refine_check(P->sc, 0, 1, none, 0, P->stream));
    return PPE_OK;
  }
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  PPE_TRY(cudaStreamIsCapturing(P->stream, &cst));
  if (cst == cudaStreamCaptureStatusActive) return capture_refine(P, mode);  // the caller builds a graph
  if (!P->prof_on) {
    PPE_TRY(cudaGraphLaunch(mode == REF_SOLVE ? P->refine_exec : P->project_exec, P->stream));
    return PPE_OK;
  }
  cudaGraphConditionalHandle none = 0;
  ppe_status s = (mode == REF_SOLVE) ? refine_probe(P, none, 0) : PPE_OK;
  bool first = true;
  while (s == PPE_OK) {
    if (!(mode == REF_PROJECT && first)) {
      int cont = 0;
      PPE_TRY(cudaMemcpyAsync(&cont, &P->sc->cont, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
      PPE_TRY(cudaStreamSynchronize(P->stream));
      if (!cont) break;
    }
    first = false;
    s = refine_body(P, mode, none, 0);
  }
  return s;
}

// Plans whose ppe_project keeps the first solve's p in FP32 (XI_F32): the FP32
// form with at least one sweep, register-staged x passes (nx/2 a power of two
// with a compiled length, 16 .. 256) and an exact inverse-transform scaling
// ((nx/2) nz a power of two).
bool p32_ok(const ppe_grid& g, const ppe_options& o) {
  const unsigned m = (unsigned)(g.nx / 2), s = m * (unsigned)g.nz;
  return o.precision == PPE_FP32_REFINE && o.max_sweeps >= 1 && m >= 16 && m <= 256 && (m & (m - 1u)) == 0u &&
         (s & (s - 1u)) == 0u;
}

// Tile sizes of the right-hand-side kernel: largest tj in {8, 4, 2, 1} whose
// shared memory lets two CTAs share an SM, else one.
void choose_rhs_tiles(ppe_plan_t P) {
  const int nx = P->g.nx;
  int tj = 2;  // measured best at 256^3 on a GB300 (register-limited occupancy)
  while (tj > 1 && (rhs_smem(nx, tj) > 110 * 1024 || tj > rhs_max_lines(nx))) tj /= 2;
  P->tj = tj;
  P->kc = P->g.nz < 8 ? P->g.nz : 8;
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
  b += (fp32 ? 16 : 8) * n;                                             // f (and p) as pairs
  if (opt && p32_ok(*g, *opt)) b += 4 * n;                              // the first solve's p in FP32
  b += 8 * (2 * n + (size_t)g->nx * (g->ny + 1) * g->nz);               // u_pre, v_pre, w_pre
  b += (fp32 ? 4 : 8) * nxh * g->nz * (size_t)g->ny + 8 * nxh * g->nz;  // upper bound of the tables
  b += 48 * (size_t)g->ny * g->nz;                                       // per-CTA partial sums
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
  o.compat_tol = 1e-12;
  o.bc_top = PPE_BC_WALL;
  if (opt) o = *opt;
  if (o.precision != PPE_FP64 && o.precision != PPE_FP32_REFINE) return PPE_ERR_INVALID_ARG;
  if (o.face_rule != PPE_FACE_ARITHMETIC && o.face_rule != PPE_FACE_HARMONIC) return PPE_ERR_INVALID_ARG;
  if (o.max_sweeps < 0 || o.max_sweeps > kMaxSweeps) return PPE_ERR_INVALID_ARG;
  if (o.precision == PPE_FP32_REFINE && !(o.refine_tol >= 0)) return PPE_ERR_INVALID_ARG;
  if (!(o.compat_tol >= 0)) return PPE_ERR_INVALID_ARG;
  if (o.bc_top != PPE_BC_WALL && o.bc_top != PPE_BC_OUTFLOW) return PPE_ERR_INVALID_ARG;

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
  // pairs round at 2^-48 per operation: lines of up to 512 points keep the
  // fields within 1e-12 of FP64 results; longer lines (and the outflow top's
  // tridiagonal solve) stay in native FP64
  P->pairs = !P->fp32 && o.bc_top == PPE_BC_WALL && g->nx <= 512 && g->ny <= 512 && g->nz <= 512;
  P->nxh = g->nx / 2 + 1;
  P->gd.nx = g->nx;
  P->gd.ny = g->ny;
  P->gd.nz = g->nz;
  P->gd.top_open = o.bc_top == PPE_BC_OUTFLOW ? 1 : 0;
  P->gd.idx = g->nx / g->lx;
  P->gd.idy = g->ny / g->ly;
  P->gd.idz = g->nz / g->lz;
  P->gd.fd_nx = make_fastdiv((uint32_t)g->nx);
  P->gd.fd_nxh = make_fastdiv((uint32_t)(g->nx / 2 + 1));
  P->gd.fd_m = make_fastdiv((uint32_t)(g->nx / 2));
  P->gd.fd_ny = make_fastdiv((uint32_t)g->ny);
  P->gd.fd_nyp1 = make_fastdiv((uint32_t)(g->ny + 1));
  const double dy = g->ly / g->ny;
  P->a_y = 1.0 / (dy * dy);
  const int maxr = P->fp32 ? 16 : 8;  // radix 16 in FP64 would need 128+ registers per butterfly
  P->rp_half = radix_plan(g->nx / 2, maxr);
  P->rp_z = radix_plan(g->nz, maxr);
  P->lpb = choose_lpb(g->nx);
  P->tkx = choose_tkx(g->nz, P->fp32, true);
  P->tky = choose_tkx(g->ny, P->fp32, false);
  P->rp_y = radix_plan(g->ny, maxr);
  P->cplx_bytes = P->fp32 ? 8 : 16;

  ppe_status s = PPE_OK;
  const size_t nspec = (size_t)P->nxh * g->ny * g->nz;
  s = alloc_status(cudaMalloc(&P->spec, nspec * P->cplx_bytes));
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->sc, sizeof(DevScalars)));
  const size_t ncell = (size_t)g->nx * g->ny * g->nz, nvf = (size_t)g->nx * (g->ny + 1) * g->nz;
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->fdf, sizeof(df) * ncell));
  if (s == PPE_OK && P->fp32) s = alloc_status(cudaMalloc((void**)&P->pdf, sizeof(df) * ncell));
  if (s == PPE_OK && p32_ok(P->g, o)) s = alloc_status(cudaMalloc((void**)&P->p32, sizeof(float) * ncell));
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->upre, sizeof(df) * ncell));
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->vpre, sizeof(df) * nvf));
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->wpre, sizeof(df) * ncell));
  if (s == PPE_OK) s = alloc_status(cudaMalloc((void**)&P->rhs_part, 3 * sizeof(double2) * g->ny * g->nz));
  P->workspace = nspec * P->cplx_bytes + sizeof(DevScalars) + (P->fp32 ? 2 : 1) * sizeof(df) * ncell +
                 (P->p32 ? sizeof(float) * ncell : 0) +
                 sizeof(df) * (2 * ncell + nvf) + P->cplx_bytes * (g->nx + g->nz) +
                 3 * sizeof(double2) * g->ny * g->nz;
  choose_rhs_tiles(P);
  if (s == PPE_OK) {
    if (P->fp32) {
      s = make_twiddles<float>(&P->tw_x, g->nx);
      if (s == PPE_OK) s = make_twiddles<float>(&P->tw_z, g->nz);
      if (s == PPE_OK) s = P->gd.top_open ? make_thomas<float>(P) : make_dct_tables<float>(P);
      // walls: the multipliers of the tridiagonal y method too (PPE_Y_TRIDIAGONAL)
      if (s == PPE_OK && !P->gd.top_open && yscan_elems(g->ny) > 0) {
        s = make_thomas<float>(P);
        P->yscan_ok = s == PPE_OK;
      }
      if (s == PPE_OK) s = cuda_status(set_smem_limits<float>());
    } else if (P->pairs) {
      s = make_twiddles<dd>(&P->tw_x, g->nx);
      if (s == PPE_OK) s = make_twiddles<dd>(&P->tw_z, g->nz);
      if (s == PPE_OK) s = make_dct_tables<dd>(P);
      if (s == PPE_OK) s = cuda_status(set_smem_limits<dd>());
    } else {
      s = make_twiddles<double>(&P->tw_x, g->nx);
      if (s == PPE_OK) s = make_twiddles<double>(&P->tw_z, g->nz);
      if (s == PPE_OK) s = make_thomas<double>(P);
      if (s == PPE_OK) s = cuda_status(set_smem_limits<double>());
    }
  }
  // the plane-layout schedules where their kernels exist (and, for the fused
  // pass, the GPU can co-schedule its clusters); LEGACY by default (measured
  // fastest at 256^3 on a GB300: 1.126 ms per projection against 1.167 ms with
  // PENCIL and 1.399 ms with FUSED), the others through ppe_set_tuning
  {
    const int M = g->nx / 2;
    const bool base_ok = s == PPE_OK && P->fp32 && !P->gd.top_open && M >= 16 && M <= 512 && (M & (M - 1)) == 0;
    if (base_ok && zyz_supported(g->ny, g->nz) && make_spec_tmap(P, &P->tmap, zyz_cols(g->ny, g->nz))) {
      int nc = 0;
      P->zyz_ok = zyz_max_clusters(P->gd, &nc) == cudaSuccess && nc > 0;
      cudaGetLastError();
    }
    if (base_ok && pencil_supported(g->ny, g->nz))
      P->pencil_ok = make_spec_tmap(P, &P->tmap_z, pencil_zcols(g->ny, g->nz));
  }
  set_sched(P, PPE_SPECTRAL_LEGACY);
  // COSINE by default: at 256^3 on a GB300 its y pass takes 58 us against 84 us
  // for the tridiagonal scans (ppe_set_tuning / the autotuner choose per grid)
  P->y_solve = PPE_Y_COSINE;
  if (s == PPE_OK && P->fp32) s = build_refine_graphs(P);
  if (s == PPE_OK) s = cuda_status(launch_init_scalars(P->sc, 1.0, o.refine_tol, 0, P->stream));
  if (s == PPE_OK)
    s = cuda_status(cudaMemcpyAsync((char*)P->sc + offsetof(DevScalars, part), &P->rhs_part, sizeof(P->rhs_part),
                                    cudaMemcpyHostToDevice, P->stream));
  // grid-only constants (1/dx^2 ...) for a ppe_solve that no ppe_rhs preceded
  if (s == PPE_OK) s = cuda_status(launch_make_const(P->gd, P->sc, 1.0, P->stream));
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
  // nothing of the plan may be in flight when its memory is freed
  if (P->acin) {
    cudaStreamSynchronize(P->acin);
    cudaStreamSynchronize(P->acout);
  }
  cudaStreamSynchronize(P->stream);
  cudaFree(P->spec);
  cudaFree(P->tw_x);
  cudaFree(P->tw_z);
  cudaFree(P->tab);
  cudaFree(P->tw_y);
  cudaFree(P->wq_y);
  cudaFree(P->lam);
  cudaFree(P->line_off);
  cudaFree(P->line_len);
  cudaFree(P->fdf);
  cudaFree(P->rhs_part);
  for (int i = 0; i < 8; ++i) cudaFree(P->vc[i]);
  cudaFree(P->pcg_part);
  if (P->pcg_exec) cudaGraphExecDestroy(P->pcg_exec);
  cudaFree(P->pdf);
  cudaFree(P->p32);
  cudaFree(P->upre);
  cudaFree(P->vpre);
  cudaFree(P->wpre);
  cudaFree(P->sc);
  if (P->refine_exec) cudaGraphExecDestroy(P->refine_exec);
  if (P->project_exec) cudaGraphExecDestroy(P->project_exec);
  for (int i = 0; i < 12; ++i) cudaFree(P->io[i]);
  for (int b = 0; b < 2; ++b) {
    for (int i = 0; i < 9; ++i) cudaFree(P->aio[b][i]);
    if (P->aev_in[b]) cudaEventDestroy(P->aev_in[b]);
    if (P->aev_done[b]) cudaEventDestroy(P->aev_done[b]);
    if (P->aev_out[b]) cudaEventDestroy(P->aev_out[b]);
  }
  if (P->acin) cudaStreamDestroy(P->acin);
  if (P->acout) cudaStreamDestroy(P->acout);
  if (P->ahsc) cudaFreeHost(P->ahsc);
  if (P->prof_ev)
    for (cudaEvent_t e : *P->prof_ev) cudaEventDestroy(e);
  delete P->prof_ev;
  delete P->prof_name;
  delete P;
}

ppe_status ppe_get_tuning(ppe_plan_t P, ppe_tuning* t) {
  if (!P || !t) return PPE_ERR_INVALID_ARG;
  t->rhs_lines = P->tj;
  t->rhs_planes = P->kc;
  t->x_lines = P->lpb;
  t->z_cols = P->tkx;
  t->y_cols = P->tky;
  t->spectral = P->sched;
  t->y_solve = P->y_solve;
  return PPE_OK;
}

ppe_status ppe_set_tuning(ppe_plan_t P, const ppe_tuning* t) {
  if (!P || !t) return PPE_ERR_INVALID_ARG;
  auto pow2 = [](int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; };
  const size_t lim = 227 * 1024;
  const int nx = P->g.nx, ny = P->g.ny, nz = P->g.nz;
  if (!pow2(t->rhs_lines, 1, 8) || rhs_smem(nx, t->rhs_lines) > rhs_smem_limit() ||
      t->rhs_lines > rhs_max_lines(nx))
    return PPE_ERR_INVALID_ARG;
  if (t->rhs_planes < 1 || t->rhs_planes > nz) return PPE_ERR_INVALID_ARG;
  if (!pow2(t->x_lines, 1, 64)) return PPE_ERR_INVALID_ARG;
  if (!pow2(t->z_cols, 1, 16) || !pow2(t->y_cols, 1, 32)) return PPE_ERR_INVALID_ARG;
  if (!sched_ok(P, t->spectral)) return PPE_ERR_INVALID_ARG;
  if (t->y_solve != PPE_Y_COSINE && !(t->y_solve == PPE_Y_TRIDIAGONAL && P->yscan_ok)) return PPE_ERR_INVALID_ARG;
  const size_t xs = P->fp32 ? (xfwd_smem<float>(nx, t->x_lines) > xinv_smem<float>(nx, t->x_lines)
                                   ? xfwd_smem<float>(nx, t->x_lines) : xinv_smem<float>(nx, t->x_lines))
                            : (xfwd_smem<double>(nx, t->x_lines) > xinv_smem<double>(nx, t->x_lines)
                                   ? xfwd_smem<double>(nx, t->x_lines) : xinv_smem<double>(nx, t->x_lines));
  const size_t zs = P->fp32 ? zfft_smem<float>(nz, t->z_cols) : zfft_smem<double>(nz, t->z_cols);
  const size_t ys = P->fp32 ? zfft_smem<float>(ny, t->y_cols) : (P->pairs ? zfft_smem<dd>(ny, t->y_cols) : 0);
  const size_t xlim = P->fp32 ? xpass_smem_limit<float>() : xpass_smem_limit<double>();
  const size_t zlim = P->fp32 ? zpass_smem_limit<float>() : zpass_smem_limit<double>();
  if (xs > xlim || zs > zlim || ys > lim) return PPE_ERR_INVALID_ARG;
  PPE_TRY(cudaStreamSynchronize(P->stream));
  if (P->pcg_exec) {  // rebuilt with the new shapes on the next unsplit call
    cudaGraphExecDestroy(P->pcg_exec);
    P->pcg_exec = nullptr;
  }
  ppe_tuning prev;
  ppe_get_tuning(P, &prev);
  auto apply = [&](const ppe_tuning& u) {
    P->tj = u.rhs_lines;
    P->kc = u.rhs_planes;
    P->lpb = u.x_lines;
    P->tkx = u.z_cols;
    P->tky = u.y_cols;
    set_sched(P, u.spectral);
    P->y_solve = u.y_solve;
    return P->fp32 ? build_refine_graphs(P) : PPE_OK;
  };
  const ppe_status s = apply(*t);
  if (s != PPE_OK) apply(prev);  // the plan keeps its previous shapes and graphs
  return s;
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
  NvtxRange _nvtx("ppe_rhs");
  if (!P || !u || !v || !w || !S || !rho || !p_n || !p_nm1 || !f || !(dt > 0)) return PPE_ERR_INVALID_ARG;
  StencilIn in = make_in(P, u, v, w, S, rho, p_n, p_nm1, dt);
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  PPE_LAUNCH(P, K_INIT, launch_init_scalars(P->sc, rho0, P->opt.refine_tol, 0, P->stream));
  if (!(rho0 > 0)) PPE_LAUNCH(P, K_RHO_MIN, launch_rho_min(rho, n, P->sc, P->stream));
  PPE_LAUNCH(P, K_CONST, launch_make_const(P->gd, P->sc, dt, P->stream));
  PPE_LAUNCH(P, K_RHS, launch_rhs(P->gd, in, P->sc, f, nullptr, nullptr, nullptr, nullptr, P->tj, P->kc, P->stream));
  PPE_TRY(launch_finish_sums(P->gd, P->sc, P->stream));
  return PPE_OK;
}

ppe_status ppe_solve(ppe_plan_t P, const double* f, double* p) {
  NvtxRange _nvtx("ppe_solve");
  if (!P || !f || !p) return PPE_ERR_INVALID_ARG;
  StencilIn in;
  memset(&in, 0, sizeof(in));
  in.f = f;
  PPE_LAUNCH(P, K_INIT, launch_init_scalars(P->sc, -1.0, P->opt.refine_tol, 1, P->stream));
  ppe_status s;
  if (P->fp32) {
    PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<float>(SRC_F, true, P->gd, in, P->sc, 0, P->fdf, nullptr,
                                               (cpx<float>*)P->spec, P->rp_half, (const cpx<float>*)P->tw_x, P->lpb,
                                               P->stream));
    if ((s = solve_tail<float>(P, XI_DF, nullptr, P->pdf, false)) != PPE_OK) return s;
    if ((s = refine(P, REF_SOLVE)) != PPE_OK) return s;
    PPE_LAUNCH(P, K_DF_TO_D,
               launch_df_to_d(P->pdf, p, (size_t)P->g.nx * P->g.ny * P->g.nz, P->stream));
    return PPE_OK;
  }
  return with_fp64_type(P, [&](auto tag) -> ppe_status {
    using T = decltype(tag);
    PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<T>(SRC_F, true, P->gd, in, P->sc, 0, nullptr, nullptr, (cpx<T>*)P->spec,
                                           P->rp_half, (const cpx<T>*)P->tw_x, P->lpb, P->stream));
    return solve_tail<T>(P, XI_F64, p, nullptr, false);
  });
}

ppe_status ppe_correct(ppe_plan_t P, const double* u, const double* v, const double* w, const double* rho,
                       const double* p, const double* p_n, const double* p_nm1, double rho0, double dt,
                       double* u_out, double* v_out, double* w_out) {
  NvtxRange _nvtx("ppe_correct");
  if (!P || !u || !v || !w || !rho || !p || !p_n || !p_nm1 || !u_out || !v_out || !w_out || !(dt > 0))
    return PPE_ERR_INVALID_ARG;
  StencilIn in = make_in(P, u, v, w, nullptr, rho, p_n, p_nm1, dt);
  in.p = p;
  if (rho0 > 0) PPE_TRY(launch_set_rho0(P->sc, rho0, P->stream));
  PPE_LAUNCH(P, K_CONST, launch_make_const(P->gd, P->sc, dt, P->stream));
  PPE_LAUNCH(P, K_CORRECT, launch_correct_full(P->gd, in, P->sc, u_out, v_out, w_out, P->stream));
  return PPE_OK;
}

ppe_status ppe_project(ppe_plan_t P, const ppe_fields* F) {
  NvtxRange _nvtx("ppe_project");
  if (!P || !F || !F->u || !F->v || !F->w || !F->S || !F->rho || !F->p_n || !F->p_nm1 || !F->p || !F->u_out ||
      !F->v_out || !F->w_out || !(F->dt > 0))
    return PPE_ERR_INVALID_ARG;
  StencilIn in = make_in(P, F->u, F->v, F->w, F->S, F->rho, F->p_n, F->p_nm1, F->dt);
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  PPE_LAUNCH(P, K_INIT, P->fp32 ? launch_init_scalars(P->sc, F->rho0, P->opt.refine_tol, 0, P->stream, F->p,
                                                       F->u_out, F->v_out, F->w_out)
                                 : launch_init_scalars(P->sc, F->rho0, P->opt.refine_tol, 0, P->stream));
  if (!(F->rho0 > 0)) PPE_LAUNCH(P, K_RHO_MIN, launch_rho_min(F->rho, n, P->sc, P->stream));
  PPE_LAUNCH(P, K_CONST, launch_make_const(P->gd, P->sc, F->dt, P->stream));
  ppe_status s;
  if (P->fp32) {
    PPE_LAUNCH(P, K_RHS, launch_rhs(P->gd, in, P->sc, F->f, P->fdf, P->upre, P->vpre, P->wpre, P->tj, P->kc,
                                    P->stream));
    PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<float>(SRC_FDF, true, P->gd, in, P->sc, 0, P->fdf, nullptr,
                                               (cpx<float>*)P->spec, P->rp_half, (const cpx<float>*)P->tw_x, P->lpb,
                                               P->stream));
    // the first solve's p: in FP32 where the first sweep reads it so (p32), else as pairs
    if ((s = solve_tail<float>(P, P->p32 ? XI_F32 : XI_DF, nullptr, P->pdf, false, true, P->p32)) != PPE_OK)
      return s;
    if ((s = refine(P, REF_PROJECT)) != PPE_OK) return s;
  } else {
    PPE_LAUNCH(P, K_RHS, launch_rhs(P->gd, in, P->sc, F->f, P->fdf, P->upre, P->vpre, P->wpre, P->tj, P->kc,
                                    P->stream));
    s = with_fp64_type(P, [&](auto tag) -> ppe_status {
      using T = decltype(tag);
      PPE_LAUNCH(P, K_XFWD_F, launch_xfwd<T>(SRC_FDF, true, P->gd, in, P->sc, 0, P->fdf, nullptr, (cpx<T>*)P->spec,
                                             P->rp_half, (const cpx<T>*)P->tw_x, P->lpb, P->stream));
      return solve_tail<T>(P, XI_F64, F->p, nullptr, false);
    });
    if (s != PPE_OK) return s;
    PPE_LAUNCH(P, K_CORRECT, launch_correct_pre(P->gd, F->dt, P->upre, P->vpre, P->wpre, nullptr, F->p, P->sc,
                                                F->u_out, F->v_out, F->w_out, P->stream));
  }
  return PPE_OK;
}

ppe_status ppe_project_unsplit(ppe_plan_t P, const ppe_fields* F, double tol, int max_iter) {
  NvtxRange _nvtx("ppe_project_unsplit");
  if (!P || !F || !F->u || !F->v || !F->w || !F->S || !F->rho || !F->p || !F->u_out || !F->v_out || !F->w_out ||
      !(F->dt > 0) || !(tol >= 0) || max_iter < 0 || max_iter > 100000)
    return PPE_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  PPE_TRY(cudaStreamIsCapturing(P->stream, &cst));
  if (cst != cudaStreamCaptureStatusNone) return PPE_ERR_INVALID_ARG;  // not capturable
  if (P->gd.top_open) return PPE_ERR_INVALID_ARG;  // the unsplit baseline has walls only
  ppe_status s = ensure_vc(P);
  if (s != PPE_OK) return s;
  if (!P->pcg_exec && (s = build_pcg_graph(P)) != PPE_OK) return s;
  const VcConst C = make_vc_const(P->g, F->dt);
  df** V = P->vc;
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  PPE_LAUNCH(P, K_INIT, launch_init_scalars(P->sc, 1.0, P->opt.refine_tol, 0, P->stream));
  PPE_TRY(cudaMemsetAsync(V[VC_X], 0, sizeof(df) * n, P->stream));
  PPE_TRY(cudaMemsetAsync(V[VC_P], 0, sizeof(df) * n, P->stream));  // p0 = 0 p - zs needs finite p
  PPE_LAUNCH(P, K_VC_SETUP, launch_vc_setup(P->gd, P->opt.face_rule, F->u, F->v, F->w, F->S, F->rho, C, V[VC_AX],
                                            V[VC_AY], V[VC_AZ], V[VC_R], P->sc, P->pcg_part, P->stream));
  PPE_LAUNCH(P, K_VC_SCALAR, launch_vc_start(P->gd, P->sc, P->pcg_part, tol, max_iter, P->stream));
  // z0 = M^{-1} r0, rz0, p0 = z0
  if ((s = vc_precond(P)) != PPE_OK) return s;
  PPE_LAUNCH(P, K_VC_DOTS, launch_vc_dots(P->gd, V[VC_R], V[VC_ZS], V[VC_R], P->pcg_part, P->stream));
  cudaGraphConditionalHandle none = 0;
  PPE_LAUNCH(P, K_VC_SCALAR, launch_vc_beta(P->gd, P->sc, P->pcg_part, 1, none, 0, P->stream));
  PPE_LAUNCH(P, K_VC_PUPDATE, launch_vc_pupdate(P->gd, V[VC_P], V[VC_ZS], P->sc, P->stream));
  if (max_iter > 0) {
    if (!P->prof_on) {
      PPE_TRY(cudaGraphLaunch(P->pcg_exec, P->stream));
    } else {
      // per-kernel timing: the same iteration driven from the host
      for (;;) {
        int cont = 0;
        PPE_TRY(cudaMemcpyAsync(&cont, &P->sc->pcg_cont, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
        PPE_TRY(cudaStreamSynchronize(P->stream));
        if (!cont) break;
        if ((s = vc_iteration(P, none, 0)) != PPE_OK) return s;
      }
    }
  }
  PPE_LAUNCH(P, K_VC_CORRECT, launch_vc_correct(P->gd, F->u, F->v, F->w, V[VC_X], V[VC_AX], V[VC_AY], V[VC_AZ], C,
                                                P->sc, P->pcg_part, F->p, F->u_out, F->v_out, F->w_out,
                                                P->stream));
  return PPE_OK;
}

ppe_status ppe_divergence_constraint(ppe_plan_t P, const double* C, const double* comp_g, const double* comp_l,
                                     const double* mdot, const double* rho_g, const double* rho_l,
                                     const unsigned char* under_resolved, double* S, double* rho) {
  if (!P || !C || !comp_g || !comp_l || !mdot || !rho_g || !rho_l || !S) return PPE_ERR_INVALID_ARG;
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  PPE_LAUNCH(P, K_DIV_S, launch_div_constraint(n, C, comp_g, comp_l, mdot, rho_g, rho_l, under_resolved, S, rho,
                                               P->stream));
  return PPE_OK;
}

ppe_status ppe_unsplit_info(ppe_plan_t P, int* iterations, double* rel_residual) {
  if (!P || !iterations || !rel_residual) return PPE_ERR_INVALID_ARG;
  DevScalars h;
  PPE_TRY(cudaMemcpyAsync(&h, P->sc, sizeof(h), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaStreamSynchronize(P->stream));
  *iterations = h.pcg_iter;
  *rel_residual = h.pcg_rel;
  return (h.pcg_rel <= h.pcg_tol) ? PPE_OK : PPE_ERR_NOT_CONVERGED;
}

struct ppe_batch_s {
  cudaGraphExec_t exec;
  cudaStream_t stream;
  int n;
  int form;            // PPE_BATCH_GRAPH or PPE_BATCH_PERSISTENT
  void* dev;           // persistent form: grids, items, stage tiles, counters, stop marks, control block
  BatchCtl* ctl;
  long long nitems;
  int ctas;
};

namespace {

// A plan and its fields that the persistent batched kernel can run.
bool batch_plan_ok(ppe_plan_t P) {
  return P->fp32 && !P->gd.top_open && P->sched == PPE_SPECTRAL_LEGACY && P->opt.max_sweeps >= 1 &&
         P->opt.max_sweeps <= kMaxSweeps && batch_dims_ok(P->g.nx, P->g.ny, P->g.nz);
}

bool fields_ok(const ppe_fields* F) {
  return F->u && F->v && F->w && F->S && F->rho && F->p_n && F->p_nm1 && F->p && F->u_out && F->v_out &&
         F->w_out && F->dt > 0;
}

size_t align_up(size_t b) { return (b + 255) & ~(size_t)255; }

// Builds the persistent form of a batch into B (B->stream set): the grid
// descriptors, the two queues (the whole projection; a further sweep), the
// device state, and a graph: reset, persistent launch, then WHILE (a loop test
// asked for another sweep) { sweep reset, persistent launch of the sweep queue }.
ppe_status batch_persistent(ppe_batch_t B, int n, const ppe_plan_t* plans, const ppe_fields* fields,
                            const ppe_batch_options& o) {
  std::vector<int> nx(n), ny(n), nz(n), rg(n);
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    ppe_plan_t P = plans[i];
    nx[i] = P->g.nx;
    ny[i] = P->g.ny;
    nz[i] = P->g.nz;
    rg[i] = fields[i].rho0 > 0 ? 1 : 0;
    smem = std::max(smem, batch_smem(nx[i], ny[i], nz[i]));
  }
  const long grain = o.grain > 0 ? o.grain : 65536;
  const long long n_full = batch_item_count(n, nx.data(), ny.data(), nz.data(), rg.data(), 0, grain);
  const long long n_sweep = batch_item_count(n, nx.data(), ny.data(), nz.data(), rg.data(), BS_RES, grain);
  if (n_full < 1 || n_full > 0x7FFFFFFFll) return PPE_ERR_INVALID_ARG;
  const int ndone = kBatchStages * n;
  std::vector<BatchItem> full((size_t)n_full), sweep((size_t)n_sweep);
  std::vector<unsigned> need(ndone), tiles(ndone);
  const int window = o.window > 0 ? o.window : n;
  const int stagger = o.stagger >= 0 ? o.stagger : 2;
  batch_schedule(n, nx.data(), ny.data(), nz.data(), rg.data(), window, stagger, 0, grain, full.data(), need.data(),
                 tiles.data());
  batch_schedule(n, nx.data(), ny.data(), nz.data(), rg.data(), window, stagger, BS_RES, grain, sweep.data(),
                 need.data(), tiles.data());
  std::vector<BatchGrid> grids(n);
  for (int i = 0; i < n; ++i) {
    ppe_plan_t P = plans[i];
    const ppe_fields* F = &fields[i];
    BatchGrid& G = grids[i];
    memset(&G, 0, sizeof(G));
    G.g = P->gd;
    G.in = make_in(P, F->u, F->v, F->w, F->S, F->rho, F->p_n, F->p_nm1, F->dt);
    G.sc = P->sc;
    G.f64 = F->f;
    G.fdf = P->fdf;
    G.pdf = P->pdf;
    G.upre = P->upre;
    G.vpre = P->vpre;
    G.wpre = P->wpre;
    G.spec = (cpx<float>*)P->spec;
    G.tw_x = (const cpx<float>*)P->tw_x;
    G.tw_z = (const cpx<float>*)P->tw_z;
    G.tw_y = (const cpx<float>*)P->tw_y;
    G.wq_y = (const cpx<float>*)P->wq_y;
    const float* lam = (const float*)P->lam;
    G.lam_x = lam;
    G.lam_y = lam + P->nxh;
    G.lam_z = lam + P->nxh + P->g.ny;
    G.out_p = F->p;
    G.out_u = F->u_out;
    G.out_v = F->v_out;
    G.out_w = F->w_out;
    G.rho0 = F->rho0;
    G.tol = P->opt.refine_tol;
    G.scale = 1.0 / ((double)(P->g.nx / 2) * (double)P->g.nz);
    G.smax = P->opt.max_sweeps;
    G.lpb = batch_lpb(P->g.nx);
    G.tkx = batch_tkx(P->g.nz, true);
    G.tky = batch_tkx(P->g.ny, false);
    G.kc = P->g.nz < 8 ? P->g.nz : 8;
    G.stage0 = kBatchStages * i;
  }
  // one allocation: grids | full queue | sweep queue | need | tiles | done (+ sentinel) | stop | ctl
  const size_t o_full = align_up(sizeof(BatchGrid) * n);
  const size_t o_sweep = o_full + align_up(sizeof(BatchItem) * (size_t)n_full);
  const size_t o_need = o_sweep + align_up(sizeof(BatchItem) * (size_t)n_sweep);
  const size_t o_tiles = o_need + align_up(sizeof(unsigned) * ndone);
  const size_t o_done = o_tiles + align_up(sizeof(unsigned) * ndone);
  const size_t o_stop = o_done + align_up(sizeof(unsigned) * (ndone + 1));
  const size_t o_ctl = o_stop + align_up(sizeof(int) * n);
  const size_t total = o_ctl + align_up(sizeof(BatchCtl));
  char* d = nullptr;
  cudaError_t e = cudaMalloc(&d, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return alloc_status(e);
  }
  B->dev = d;
  B->ctl = (BatchCtl*)(d + o_ctl);
  B->nitems = n_full;
  PPE_TRY(cudaMemcpy(d, grids.data(), sizeof(BatchGrid) * n, cudaMemcpyHostToDevice));
  PPE_TRY(cudaMemcpy(d + o_full, full.data(), sizeof(BatchItem) * (size_t)n_full, cudaMemcpyHostToDevice));
  PPE_TRY(cudaMemcpy(d + o_sweep, sweep.data(), sizeof(BatchItem) * (size_t)n_sweep, cudaMemcpyHostToDevice));
  PPE_TRY(cudaMemcpy(d + o_need, need.data(), sizeof(unsigned) * ndone, cudaMemcpyHostToDevice));
  PPE_TRY(cudaMemcpy(d + o_tiles, tiles.data(), sizeof(unsigned) * ndone, cudaMemcpyHostToDevice));
  PPE_TRY(cudaMemset(d + o_ctl, 0, sizeof(BatchCtl)));
  int occ = 0, dev = 0, sms = 0;
  PPE_TRY(batch_occupancy(smem, &occ));
  PPE_TRY(cudaGetDevice(&dev));
  PPE_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (occ < 1) return PPE_ERR_INVALID_ARG;  // the largest stage's tile does not fit an SM
  const int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, occ) : occ;
  B->ctas = per_sm * sms;
  const double ws = o.wait_seconds > 0 ? o.wait_seconds : 2.0;
  const unsigned long long wait_ns = (unsigned long long)(ws * 1e9);
  const BatchGrid* dg = (const BatchGrid*)d;
  unsigned* done = (unsigned*)(d + o_done);
  const unsigned* dneed = (const unsigned*)(d + o_need);
  const unsigned* dtiles = (const unsigned*)(d + o_tiles);
  int* stop = (int*)(d + o_stop);
  // capture
  cudaStream_t cs = nullptr, bs = nullptr;
  cudaGraph_t g = nullptr;
  ppe_status st = PPE_OK;
  bool cap = false, bcap = false;
  auto ok = [&](cudaError_t r) {
    if (r != cudaSuccess && st == PPE_OK) st = PPE_ERR_CUDA;
    return st == PPE_OK;
  };
  if (ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) &&
      ok(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking)) &&
      ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal))) {
    cap = true;
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t cond = nullptr;
    cudaGraphNodeParams cp = {};
    if (ok(launch_batch_reset(dg, n, done, ndone, stop, B->ctl, cs)) &&
        ok(launch_batch(dg, n, (const BatchItem*)(d + o_full), (int)n_full, done, ndone, dneed, dtiles, stop,
                        B->ctl, wait_ns, o.test_unset_wait ? 1 : 0, B->ctas, smem, cs)) &&
        ok(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps)) &&
        ok(cudaGraphConditionalHandleCreate(&h, cg, 0u, cudaGraphCondAssignDefault)) &&
        ok(launch_batch_cond(B->ctl, h, cs)) &&
        ok(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps))) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      if (ok(cudaGraphAddNode(&cond, cg, deps, nullptr, ndeps, &cp)) &&
          ok(cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies)) &&
          ok(cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal))) {
        bcap = true;
        if (ok(launch_batch_sweep_reset(dg, n, done, B->ctl, bs)))
          if (ok(launch_batch(dg, n, (const BatchItem*)(d + o_sweep), (int)n_sweep, done, ndone, dneed, dtiles,
                              stop, B->ctl, wait_ns, 0, B->ctas, smem, bs)))
            ok(launch_batch_cond(B->ctl, h, bs));
      }
    }
    if (bcap) {
      cudaGraph_t bg = nullptr;
      ok(cudaStreamEndCapture(bs, &bg));
    }
  }
  if (cap) ok(cudaStreamEndCapture(cs, &g));
  if (st == PPE_OK) ok(cudaGraphInstantiate(&B->exec, g, 0));
  if (g) cudaGraphDestroy(g);
  if (bs) cudaStreamDestroy(bs);
  if (cs) cudaStreamDestroy(cs);
  if (st != PPE_OK) cudaGetLastError();
  return st;
}

// Graph form: every projection captured as branches of one graph.
ppe_status batch_graph(ppe_batch_t B, int n, const ppe_plan_t* plans, const ppe_fields* fields) {
  const int nb = n < 16 ? n : 16;  // branch streams: solves on one stream run in order
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> bs(nb, nullptr);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  cudaGraph_t g = nullptr;
  ppe_status st = PPE_OK;
  bool capturing = false;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) st = PPE_ERR_CUDA;
  for (int b = 0; st == PPE_OK && b < nb; ++b)
    if (cudaStreamCreateWithFlags(&bs[b], cudaStreamNonBlocking) != cudaSuccess) st = PPE_ERR_CUDA;
  for (int b = 0; st == PPE_OK && b <= nb; ++b)
    if (cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming) != cudaSuccess) st = PPE_ERR_CUDA;
  if (st == PPE_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = PPE_ERR_CUDA;
  capturing = st == PPE_OK;
  if (st == PPE_OK && cudaEventRecord(ev[nb], cs) != cudaSuccess) st = PPE_ERR_CUDA;
  for (int b = 0; st == PPE_OK && b < nb; ++b)
    if (cudaStreamWaitEvent(bs[b], ev[nb], 0) != cudaSuccess) st = PPE_ERR_CUDA;
  // branches balanced by cells: largest grid first, each to the branch with the
  // least work so far (a branch runs its projections in order, so the most
  // loaded one sets the batch's tail)
  std::vector<int> order(n), branch(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto cells = [&](int i) { return (double)plans[i]->g.nx * plans[i]->g.ny * plans[i]->g.nz; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cells(a) > cells(b); });
  std::vector<double> load(nb, 0.0);
  for (int i : order) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch[i] = b;
    load[b] += cells(i);
  }
  for (int k = 0; st == PPE_OK && k < n; ++k) {
    const int i = order[k];
    ppe_plan_t P = plans[i];
    cudaStream_t saved = P->stream;
    P->stream = bs[branch[i]];
    st = ppe_project(P, &fields[i]);
    P->stream = saved;
  }
  for (int b = 0; st == PPE_OK && b < nb; ++b) {
    if (cudaEventRecord(ev[b], bs[b]) != cudaSuccess || cudaStreamWaitEvent(cs, ev[b], 0) != cudaSuccess)
      st = PPE_ERR_CUDA;
  }
  if (capturing) {
    cudaGraph_t cg = nullptr;
    if (cudaStreamEndCapture(cs, &cg) != cudaSuccess && st == PPE_OK) st = PPE_ERR_CUDA;
    g = cg;
  }
  if (st == PPE_OK && cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) st = PPE_ERR_CUDA;
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : bs)
    if (s) cudaStreamDestroy(s);
  if (cs) cudaStreamDestroy(cs);
  if (g) cudaGraphDestroy(g);
  if (st != PPE_OK) cudaGetLastError();
  return st;
}

}  // namespace

ppe_status ppe_batch_create_ex(ppe_batch_t* out, int n, const ppe_plan_t* plans, const ppe_fields* fields,
                               void* stream, const ppe_batch_options* opt) {
  if (!out || n < 1 || !plans || !fields) return PPE_ERR_INVALID_ARG;
  *out = nullptr;
  ppe_batch_options o;
  memset(&o, 0, sizeof(o));
  o.stagger = -1;
  if (opt) o = *opt;
  if (o.form < PPE_BATCH_AUTO || o.form > PPE_BATCH_PERSISTENT || o.ctas_per_sm < 0 || !(o.wait_seconds >= 0) ||
      o.grain < 0)
    return PPE_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return PPE_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return PPE_ERR_INVALID_ARG;
  }
  bool persistent_ok = n <= 65535;
  for (int i = 0; i < n && persistent_ok; ++i)
    persistent_ok = batch_plan_ok(plans[i]) && fields_ok(&fields[i]);
  if (o.form == PPE_BATCH_PERSISTENT && !persistent_ok) return PPE_ERR_INVALID_ARG;
  ppe_batch_t B = new (std::nothrow) ppe_batch_s;
  if (!B) return PPE_ERR_OUT_OF_MEMORY;
  memset(B, 0, sizeof(*B));
  B->stream = (cudaStream_t)stream;
  B->n = n;
  // AUTO: the graph form, which ran faster than the persistent form on every
  // batch measured on a GB300 (one 256^3 grid, 8 x 128^3, 64 x 64^3, 64
  // uneven grids)
  const bool persistent = o.form == PPE_BATCH_PERSISTENT;
  B->form = persistent ? PPE_BATCH_PERSISTENT : PPE_BATCH_GRAPH;
  const ppe_status st = persistent ? batch_persistent(B, n, plans, fields, o) : batch_graph(B, n, plans, fields);
  if (st != PPE_OK) {
    ppe_batch_destroy(B);
    return st;
  }
  *out = B;
  return PPE_OK;
}

ppe_status ppe_batch_create(ppe_batch_t* out, int n, const ppe_plan_t* plans, const ppe_fields* fields,
                            void* stream) {
  ppe_batch_options o;
  memset(&o, 0, sizeof(o));
  o.form = PPE_BATCH_GRAPH;
  o.stagger = -1;
  return ppe_batch_create_ex(out, n, plans, fields, stream, &o);
}

ppe_status ppe_batch_launch(ppe_batch_t B) {
  NvtxRange _nvtx("ppe_batch_launch");
  if (!B || !B->exec) return PPE_ERR_INVALID_ARG;
  PPE_TRY(cudaGraphLaunch(B->exec, B->stream));
  return PPE_OK;
}

ppe_status ppe_batch_status(ppe_batch_t B, int* form, long long* items, int* ctas, int* launches, int* err_grid,
                            int* err_stage) {
  if (!B) return PPE_ERR_INVALID_ARG;
  if (form) *form = B->form;
  if (items) *items = B->nitems;
  if (ctas) *ctas = B->ctas;
  if (launches) *launches = 0;
  if (err_grid) *err_grid = -1;
  if (err_stage) *err_stage = -1;
  PPE_TRY(cudaStreamSynchronize(B->stream));
  if (!B->ctl) return PPE_OK;
  BatchCtl h;
  PPE_TRY(cudaMemcpy(&h, B->ctl, sizeof(h), cudaMemcpyDeviceToHost));
  if (launches) *launches = h.launches;
  if (err_grid) *err_grid = h.err_grid;
  if (err_stage) *err_stage = h.err_stage;
  return h.status == 0 ? PPE_OK : (ppe_status)h.status;
}

void ppe_batch_destroy(ppe_batch_t B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->dev) cudaFree(B->dev);
  delete B;
}

long long ppe_batch_schedule(int n, const int* dims, const int* rho_given, int window, int stagger, int grain,
                             int first, int* out, long long cap, int* need, int* tiles) {
  if (n < 1 || !dims || !rho_given || cap < 0 || (cap > 0 && !out) || grain < 0 || (first != 0 && first != BS_RES))
    return -1;
  std::vector<int> nx(n), ny(n), nz(n), rg(n);
  for (int i = 0; i < n; ++i) {
    nx[i] = dims[3 * i];
    ny[i] = dims[3 * i + 1];
    nz[i] = dims[3 * i + 2];
    rg[i] = rho_given[i] ? 1 : 0;
    if (!batch_dims_ok(nx[i], ny[i], nz[i])) return -1;
  }
  const long gr = grain > 0 ? grain : 65536;
  const long long nitems = batch_item_count(n, nx.data(), ny.data(), nz.data(), rg.data(), first, gr);
  std::vector<BatchItem> items((size_t)nitems);
  std::vector<unsigned> nd((size_t)kBatchStages * n), nt((size_t)kBatchStages * n);
  batch_schedule(n, nx.data(), ny.data(), nz.data(), rg.data(), window > 0 ? window : n, stagger >= 0 ? stagger : 2,
                 first, gr, items.data(), nd.data(), nt.data());
  const long long m = cap < nitems ? cap : nitems;
  for (long long i = 0; i < m; ++i) {
    out[4 * i] = items[i].grid;
    out[4 * i + 1] = items[i].stage;
    out[4 * i + 2] = (int)items[i].tile0;
    out[4 * i + 3] = items[i].count;
  }
  for (size_t i = 0; i < nd.size(); ++i) {
    if (need) need[i] = (int)nd[i];
    if (tiles) tiles[i] = (int)nt[i];
  }
  return nitems;
}

ppe_status ppe_project_batched(int n, const ppe_plan_t* plans, const ppe_fields* fields, void* stream) {
  ppe_batch_t B = nullptr;
  ppe_status s = ppe_batch_create(&B, n, plans, fields, stream);
  if (s != PPE_OK) return s;
  s = ppe_batch_launch(B);
  if (s == PPE_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) s = PPE_ERR_CUDA;
  ppe_batch_destroy(B);
  return s;
}

ppe_status ppe_project_host(ppe_plan_t P, const ppe_fields* H) {
  NvtxRange _nvtx("ppe_project_host");
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
  ppe_info info;
  return ppe_get_info(P, &info);  // synchronises; device-side status (convergence, compatibility)
}

namespace {
// The report and status of one projection from a host copy of its scalars.
ppe_status info_from(ppe_plan_t P, const DevScalars& h, ppe_info* info) {
  const double fmax = h.fmax_bits ? __builtin_bit_cast(double, h.fmax_bits) : 0.0;
  const bool timed_out = h.dev_err != 0;  // a bounded device-side wait ran out (bulk copy or batch stage)
  info->f_max = fmax;
  info->rho0 = __builtin_bit_cast(double, h.rho0_bits);
  bool incompatible = false;
  const double n = (double)P->g.nx * P->g.ny * P->g.nz;
  const double idy = P->g.ny / P->g.ly;
  info->s_absmax = info->wall_flux_mean = info->wall_vmax = info->s_mean = NAN;
  info->f_mean_removed = h.f_ran ? h.f_sum / n : NAN;
  if (h.rhs_ran) {
    info->wall_flux_mean = h.wall_flux * idy / n;
    info->s_absmax = h.smax_bits ? __builtin_bit_cast(double, h.smax_bits) : 0.0;
    info->wall_vmax = h.wallv_bits ? __builtin_bit_cast(double, h.wallv_bits) : 0.0;
    // Over the cells, sum D u* = sum over (i, k) of (v*(ny) - v*(0)) / dy (x, z
    // periodic) and sum D(beta G p_hat) = 0 (G = 0 on the walls), so by Eq. (34)
    // mean(S) = wall_flux_mean - (dt/rho_0) mean(f).
    // (walls only: an open top face carries flux of both terms)
    if (h.f_ran && !P->gd.top_open) info->s_mean = info->wall_flux_mean - info->f_mean_removed / df2d(h.K.c);
  }
  // the Neumann problem needs mean(f) = 0; what the solve drops, relative to ||f||
  // (an open top has no compatibility condition)
  if (h.f_ran && P->opt.compat_tol > 0 && !P->gd.top_open) incompatible = fabs(h.f_sum / n) > P->opt.compat_tol * fmax;
  if (P->fp32) {
    // max_sweeps = 0 applies no correction; the device test that follows the
    // fused correction-and-residual kernel counts that pass as one sweep
    info->sweeps = P->opt.max_sweeps == 0 ? 0 : h.sweeps;
    if (h.last_slot >= 0 && fmax > 0)
      info->rel_residual = __builtin_bit_cast(double, h.rmax_bits[h.last_slot]) / fmax;
    else
      info->rel_residual = -1.0;
    if (timed_out) return PPE_ERR_TIMEOUT;
    if (h.last_slot >= 0 && !h.done) return PPE_ERR_NOT_CONVERGED;
  } else {
    info->sweeps = 0;
    info->rel_residual = -1.0;
  }
  return incompatible ? PPE_ERR_INCOMPATIBLE_RHS : PPE_OK;
}
}  // namespace

namespace {
// Retire the call that used staging set b: wait for its output copies and fold
// its status into the pipeline's.
ppe_status async_retire(ppe_plan_t P, int b) {
  if (!P->abusy[b]) return PPE_OK;
  PPE_TRY(cudaEventSynchronize(P->aev_out[b]));
  P->abusy[b] = 0;
  ppe_info info;
  const ppe_status st = info_from(P, P->ahsc[b], &info);
  if (P->astatus == PPE_OK) P->astatus = st;
  return PPE_OK;
}
}  // namespace

ppe_status ppe_project_host_async(ppe_plan_t P, const ppe_fields* H) {
  NvtxRange _nvtx("ppe_project_host_async");
  if (!P || !H || !H->u || !H->v || !H->w || !H->S || !H->rho || !H->p_n || !H->p_nm1 || !H->p || !H->u_out ||
      !H->v_out || !H->w_out || !(H->dt > 0))
    return PPE_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cst;
  if (cudaStreamIsCapturing(P->stream, &cst) != cudaSuccess || cst != cudaStreamCaptureStatusNone)
    return PPE_ERR_INVALID_ARG;
  const size_t n = (size_t)P->g.nx * P->g.ny * P->g.nz;
  const size_t nv = (size_t)P->g.nx * (P->g.ny + 1) * P->g.nz;
  const size_t sizes[9] = {n, nv, n, n, n, n, n, n, n};  // u v w S rho p_n p_nm1 p f
  if (!P->acin) {
    PPE_TRY(cudaStreamCreateWithFlags(&P->acin, cudaStreamNonBlocking));
    PPE_TRY(cudaStreamCreateWithFlags(&P->acout, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      PPE_TRY(cudaEventCreateWithFlags(&P->aev_in[b], cudaEventDisableTiming));
      PPE_TRY(cudaEventCreateWithFlags(&P->aev_done[b], cudaEventDisableTiming));
      PPE_TRY(cudaEventCreateWithFlags(&P->aev_out[b], cudaEventDisableTiming));
    }
    ppe_status s = alloc_status(cudaMallocHost((void**)&P->ahsc, 2 * sizeof(DevScalars)));
    if (s != PPE_OK) return s;
  }
  const int b = P->aset;
  ppe_status s = async_retire(P, b);  // the set's previous call must have left it
  if (s != PPE_OK) return s;
  const int nbuf = H->f ? 9 : 8;
  for (int i = 0; i < nbuf; ++i)
    if (!P->aio[b][i]) {
      s = alloc_status(cudaMalloc((void**)&P->aio[b][i], sizes[i] * sizeof(double)));
      if (s != PPE_OK) return s;
    }
  double** io = P->aio[b];
  // inputs on the copy-in stream (after the set's previous outputs left)
  PPE_TRY(cudaStreamWaitEvent(P->acin, P->aev_out[b], 0));
  const double* src[7] = {H->u, H->v, H->w, H->S, H->rho, H->p_n, H->p_nm1};
  for (int i = 0; i < 7; ++i)
    PPE_TRY(cudaMemcpyAsync(io[i], src[i], sizes[i] * sizeof(double), cudaMemcpyHostToDevice, P->acin));
  PPE_TRY(cudaEventRecord(P->aev_in[b], P->acin));
  // the projection on the plan's stream, then its scalars to the host
  PPE_TRY(cudaStreamWaitEvent(P->stream, P->aev_in[b], 0));
  ppe_fields D;
  D.u = io[0]; D.v = io[1]; D.w = io[2]; D.S = io[3]; D.rho = io[4];
  D.p_n = io[5]; D.p_nm1 = io[6];
  D.rho0 = H->rho0;
  D.dt = H->dt;
  D.p = io[7];
  D.u_out = io[0]; D.v_out = io[1]; D.w_out = io[2];  // in place
  D.f = H->f ? io[8] : nullptr;
  s = ppe_project(P, &D);
  if (s != PPE_OK) return s;
  PPE_TRY(cudaMemcpyAsync(&P->ahsc[b], P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaEventRecord(P->aev_done[b], P->stream));
  // outputs on the copy-out stream
  PPE_TRY(cudaStreamWaitEvent(P->acout, P->aev_done[b], 0));
  PPE_TRY(cudaMemcpyAsync(H->p, D.p, n * sizeof(double), cudaMemcpyDeviceToHost, P->acout));
  PPE_TRY(cudaMemcpyAsync(H->u_out, D.u_out, n * sizeof(double), cudaMemcpyDeviceToHost, P->acout));
  PPE_TRY(cudaMemcpyAsync(H->v_out, D.v_out, nv * sizeof(double), cudaMemcpyDeviceToHost, P->acout));
  PPE_TRY(cudaMemcpyAsync(H->w_out, D.w_out, n * sizeof(double), cudaMemcpyDeviceToHost, P->acout));
  if (H->f) PPE_TRY(cudaMemcpyAsync(H->f, D.f, n * sizeof(double), cudaMemcpyDeviceToHost, P->acout));
  PPE_TRY(cudaEventRecord(P->aev_out[b], P->acout));
  P->abusy[b] = 1;
  P->aset = b ^ 1;
  return PPE_OK;
}

ppe_status ppe_host_wait(ppe_plan_t P) {
  if (!P) return PPE_ERR_INVALID_ARG;
  // oldest call first: the set after the next one to be used
  for (int q = 0; q < 2; ++q) {
    const ppe_status s = async_retire(P, P->aset ^ q);
    if (s != PPE_OK) return s;
  }
  const ppe_status st = P->astatus;
  P->astatus = PPE_OK;
  return st;
}

ppe_status ppe_get_info(ppe_plan_t P, ppe_info* info) {
  if (!P || !info) return PPE_ERR_INVALID_ARG;
  DevScalars h;
  PPE_TRY(cudaMemcpyAsync(&h, P->sc, sizeof(h), cudaMemcpyDeviceToHost, P->stream));
  PPE_TRY(cudaStreamSynchronize(P->stream));
  return info_from(P, h, info);
}

}  // extern "C"
