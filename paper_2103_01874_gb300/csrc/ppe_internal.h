// Internal declarations shared by the libppe translation units.
#pragma once
#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "dfloat.cuh"
#include "fft.cuh"

namespace ppe {

constexpr int kMaxSweeps = 16;
constexpr int kMaxDim = 1024;

// Per-call constants of the stencils as float pairs, formed once on the device
// (k_make_const) after rho_0 is known, and read by every stencil thread.
struct StencilConst {
  df c;            // rho_0 / dt
  df g;            // dt / rho_0
  df r0h;          // rho_0 / 2   (harmonic face rule)
  df r02;          // 2 rho_0     (arithmetic face rule)
  df idx, idy, idz;
  df gx, gy, gz;   // (dt/rho_0) / dx, ...
  df lx, ly, lz;   // 1/dx^2, 1/dy^2, 1/dz^2
  df cx, cy, cz;   // (rho_0/dt) dx, (rho_0/dt) dy, (rho_0/dt) dz
};

// Device-resident scalars of one plan.  Non-negative doubles are kept as their
// IEEE bit patterns so that atomicMax / atomicMin on unsigned 64-bit integers
// order them correctly.
struct DevScalars {
  unsigned long long rho0_bits;                 // rho_0 (min(rho) or the given value)
  unsigned long long fmax_bits;                 // ||f||_inf
  unsigned long long rmax_bits[kMaxSweeps + 2]; // ||f - L p||_inf measured before sweep s
  int done;                                     // refinement converged
  int iter;                                     // residual slot of the next check (1-based)
  int cont;                                     // last check asked for another correction
  int last_slot;                                // slot of the last residual checked (-1: none)
  int sweeps;                                   // sweeps run
  double tol;                                   // refinement tolerance (relative)
  StencilConst K;                               // stencil constants of the current call
  double* out_p;                                // ppe_project outputs, set per call (k_init_scalars)
  double* out_u;
  double* out_v;
  double* out_w;
  // compatibility of the right-hand side and the mean of f, which the solve
  // drops and the refinement residual leaves out
  unsigned long long smax_bits;                 // max |S| (k_rhs_march)
  unsigned long long wallv_bits;                // max |v*| on the wall faces y = 0, Ly (k_rhs_march)
  double wall_flux;                             // sum over (i, k) of v*(ny) - v*(0)
  double f_sum;                                 // sum of f over the cells
  df f_mean;                                    // f_sum / (nx ny nz) as a pair; 0 when it is rounding noise
  int rhs_ran;                                  // wall_flux, smax, wallv belong to the last assembly
  int f_ran;                                    // f_sum, f_mean belong to the current call
  int rhs_tiles, rhs_chunks;                    // tiling of the last k_rhs_march (0: none this call)
  int x_parts;                                  // CTAs of the last forward x transform of f (0: none)
  // mean of p kept at zero by the refinement: the inverse x transform that forms
  // p writes per-CTA partial sums (p_parts of them, part[2 ny nz ..]); the next
  // first z pass totals them into zmode = -sum(p) / ny, the zero-mode value of
  // the next correction's spectrum (so p + correction has zero mean)
  double zmode;
  int p_parts;
  int dev_err;                                  // device-side errors of the current call, reported as
                                                // PPE_ERR_TIMEOUT: bit 1 a bounded wait for a bulk tensor
                                                // copy ran out; bit 2 a stage wait of the batched kernel did
  // unsplit projection (k_pcg.cu): conjugate-gradient state
  double pcg_alpha, pcg_beta, pcg_rz;           // step, direction update, r . z
  double pcg_gmean;                             // mean of the right side g (kept by r)
  df pcg_gmean_df;
  df pcg_xmean_df;                              // mean of the solution, removed from p
  double pcg_rel;                               // max |r - mean g| / max |g| after the last update
  double pcg_tol;
  unsigned long long pcg_gmax_bits, pcg_rmax_bits;
  int pcg_iter, pcg_max, pcg_cont;
  double2* part;                                // per-CTA partial sums, plan workspace (3 ny nz entries):
                                                //   [0, ny nz): k_rhs_march (wall flux, wall tiles only)
                                                //   [ny nz, 2 ny nz): forward x transform (sum of f)
                                                //   [2 ny nz, 3 ny nz): inverse x transform (sum of p)
};

struct GridDev {
  int nx, ny, nz;
  int top_open;          // 1: outflow top (p = 0 on the face y = Ly, ghost p_ny = -p_{ny-1}); 0: wall
  int spec_planes;       // spectrum layout: 0 [kz][j][kx] (kx fastest); 1 [kx][kz][j] (plane layout, the fused
                         // z-y-z pass of k_zyz.cu; index kx * ny nz + line)
  double idx, idy, idz;  // 1/dx, 1/dy, 1/dz
  FastDiv fd_nx, fd_nxh, fd_m, fd_ny, fd_nyp1;  // dividers by nx, nx/2+1, nx/2, ny, ny+1
};

inline int ilog2(int v) {
  int l = 0;
  while ((1 << (l + 1)) <= v) ++l;
  return l;
}

// Inputs of the right-hand side (Eq. (34)) and of the correction (Eq. (33)).
struct StencilIn {
  const double *u, *v, *w, *S, *rho, *pn, *pnm1;
  const double* f;   // SRC_F / SRC_RESID: the right-hand side
  const double* p;   // SRC_RESID / correction: the pressure
  const float* p0f;  // SRC_RESID (FP32 register-staged pass): the first solve's p in FP32, read at the
                     // first sweep (sc->iter == 1) in place of the pairs; NULL: always the pairs
  double inv_dt;
  double dt;
  int face_rule;     // 0 arithmetic, 1 harmonic
};

enum XSource { SRC_F = 1, SRC_RESID = 2, SRC_FDF = 3 };
enum XInvMode { XI_F64 = 0, XI_DF = 1, XI_DF_ACC = 2, XI_F32 = 3 };

// ---- launchers (k_rhs.cu) ----
cudaError_t launch_rhs(const GridDev& g, const StencilIn& in, DevScalars* sc, double* f64, df* fdf, df* upre,
                       df* vpre, df* wpre, int tj, int kc, cudaStream_t st);
// Totals of the per-CTA partial sums into sc (one CTA, finish_sums); the first
// forward z pass after an x transform of f does the same in its CTA 0.
cudaError_t launch_finish_sums(const GridDev& g, DevScalars* sc, cudaStream_t st);
size_t rhs_smem(int nx, int lines);  // dynamic shared memory of the RHS kernel for a rhs_lines value
int rhs_max_lines(int nx);  // largest rhs_lines value (lines per thread stack, or per tile when nx > 256)
cudaError_t set_rhs_smem_limit();
size_t rhs_smem_limit();  // largest dynamic shared memory every k_rhs_march instance accepts
constexpr size_t kSmemPerCta = 227 * 1024;  // opt-in shared memory per CTA (static + dynamic)

// ---- unsplit projection (k_pcg.cu) ----
// Constants of the variable-coefficient operator as pairs: 1/h^2, 1/h, 1/dt, dt h.
struct VcConst {
  df ix2, iy2, iz2;
  df idx, idy, idz, idt;
  df dthx, dthy, dthz;
};
unsigned vc_grid(size_t n);  // CTAs of the flat kernels (and their partial sums)
cudaError_t launch_vc_setup(const GridDev& g, int rule, const double* u, const double* v, const double* w,
                            const double* S, const double* rho, const VcConst& C, df* ax, df* ay, df* az, df* r,
                            DevScalars* sc, double2* part, cudaStream_t st);
cudaError_t launch_vc_start(const GridDev& g, DevScalars* sc, const double2* part, double tol, int max_iter,
                            cudaStream_t st);
cudaError_t launch_vc_apply(const GridDev& g, const df* p, const df* ax, const df* ay, const df* az, df* Kp,
                            double2* part, cudaStream_t st);
cudaError_t launch_vc_alpha(const GridDev& g, DevScalars* sc, const double2* part, cudaStream_t st);
cudaError_t launch_vc_update(const GridDev& g, df* x, df* r, const df* p, const df* Kp, DevScalars* sc,
                             cudaStream_t st);
cudaError_t launch_vc_dots(const GridDev& g, const df* r, const df* zs, const df* Kp, double2* part,
                           cudaStream_t st);
cudaError_t launch_vc_beta(const GridDev& g, DevScalars* sc, const double2* part, int first,
                           cudaGraphConditionalHandle handle, int use_handle, cudaStream_t st);
cudaError_t launch_vc_pupdate(const GridDev& g, df* p, const df* zs, const DevScalars* sc, cudaStream_t st);
// Eq. (29) and p with the mean of x removed (sum x, mean, correction)
cudaError_t launch_vc_correct(const GridDev& g, const double* u, const double* v, const double* w, const df* x,
                              const df* ax, const df* ay, const df* az, const VcConst& C, DevScalars* sc,
                              double2* part, double* p_out, double* u_out, double* v_out, double* w_out,
                              cudaStream_t st);

// ---- launchers (spectral.cuh, instantiated in k_spectral_f32.cu, k_spectral_f64.cu, k_spectral_dd.cu) ----
template <typename T>
cudaError_t launch_xfwd(int src, bool do_fft, const GridDev& g, const StencilIn& in, DevScalars* sc,
                        int sweep_slot, df* fdf, const df* pdf, cpx<T>* spec, const RadixPlan& rp_half,
                        const cpx<T>* tw_x, int lpb, cudaStream_t st);
// fin: non-NULL on the first forward pass after an x transform of f: its CTA 0
// forms the totals of the partial sums (finish_sums) before its own work.
template <typename T>
cudaError_t launch_zfft(bool inverse, const GridDev& g, cpx<T>* spec, const RadixPlan& rp,
                        const cpx<T>* tw_z, int tkx, const DevScalars* sc, DevScalars* fin, cudaStream_t st);
// y passes of the FP32 solve: zsc->zmode is the value given to the zero mode
template <typename T>
cudaError_t launch_ythomas(const GridDev& g, cpx<T>* spec, const T* tab, const int* line_off,
                           const int* line_len, T a, const DevScalars* sc, cudaStream_t st);
template <typename T>
cudaError_t launch_ydct(const GridDev& g, cpx<T>* spec, const RadixPlan& rp, const cpx<T>* tw, const cpx<T>* wq,
                        const T* lam_x, const T* lam_y, const T* lam_z, int tky, const DevScalars* zsc,
                        cudaStream_t st);
// psc non-NULL (XI_DF, XI_DF_ACC, XI_F32): the per-CTA sums of the p written go to psc->part[2 ny nz ..].
// XI_F32 (FP32 register-staged pass: nx/2 in 16 .. 256 a power of two, (nx/2) nz a power of two, so that
// the 1/((nx/2) nz) scaling is exact and the pair the XI_DF mode would store has a zero low part): p into
// p32 as FP32.  XI_DF_ACC with p32 non-NULL adds the correction to that FP32 p at the first sweep
// (psc->iter == 1), to the pairs later.
template <typename T>
cudaError_t launch_xinv(int mode, const GridDev& g, const cpx<T>* spec, double* p, df* pdf, double scale,
                        const RadixPlan& rp_half, const cpx<T>* tw_x, int lpb, const DevScalars* sc,
                        DevScalars* psc, cudaStream_t st, float* p32 = nullptr);
template <typename T>
size_t xfwd_smem(int nx, int lpb);
template <typename T>
size_t zfft_smem(int nz, int tkx);
template <typename T>
size_t xinv_smem(int nx, int lpb);
template <typename T>
cudaError_t set_smem_limits();
template <typename T>
size_t xpass_smem_limit();  // largest dynamic shared memory of the x passes (static scratch excluded)
template <typename T>
size_t zpass_smem_limit();  // the same for the z pass

// ---- tridiagonal y solve in scan form, FP32 with walls (k_yscan.cu) ----
int yscan_elems(int ny);  // elements per thread (0: ny above 512, not supported)
// zsc->zmode: the mean given to the singular line kx = kz = 0 (keeps p zero-mean)
cudaError_t launch_ythomas_scan(const GridDev& g, cpx<float>* spec, const float* tab, const int* line_off,
                                const int* line_len, float a, const DevScalars* zsc, cudaStream_t st);

// ---- fused z-y-z pass on the plane layout (k_zyz.cu) ----
bool zyz_supported(int ny, int nz);  // ny, nz in {32, 64, 128, 256}
int zyz_cols(int ny, int nz);        // j columns per CTA (the bulk tensor box width)
// largest number of co-resident clusters of the kernel for this grid (0: cannot launch)
cudaError_t zyz_max_clusters(const GridDev& g, int* n);
// tmap: 2-D map of the spectrum {ny, nz (nx/2+1)}, 8-byte elements, box {zyz_cols, nz}.
// err: dev_err of the calling plan (and zmode, the zero mode's value); fin as in launch_zfft.
cudaError_t launch_zyz(const GridDev& g, const CUtensorMap& tmap, const cpx<float>* tw_z, const cpx<float>* tw_y,
                       const cpx<float>* wq, const float* lam_x, const float* lam_y, const float* lam_z,
                       DevScalars* err, DevScalars* fin, cudaStream_t st);

// ---- bulk-copy-staged z and y passes on the plane layout (k_pencil.cu) ----
bool pencil_supported(int ny, int nz);  // ny, nz in {32, 64, 128, 256}
int pencil_zcols(int ny, int nz);       // j columns of a z tile (the tensor map's box width)
// tmap: 2-D map of the spectrum {ny, nz (nx/2+1)}, 8-byte elements, box {pencil_zcols(ny, nz), nz}
cudaError_t launch_zfft_tma(bool inverse, const GridDev& g, const CUtensorMap& tmap, const cpx<float>* tw,
                            DevScalars* err, DevScalars* fin, cudaStream_t st);
cudaError_t launch_ydct_tma(const GridDev& g, cpx<float>* spec, const cpx<float>* tw, const cpx<float>* wq,
                            const float* lam_x, const float* lam_y, const float* lam_z, DevScalars* err,
                            cudaStream_t st);  // err->zmode: the zero mode's value

// ---- persistent batched projection (k_batch.cu) ----
// One launch runs the FP32 + pair-refinement projections of many grids: a
// device work queue of (grid, stage, tile) items, taken in order by resident
// CTAs; a stage of a grid starts once every tile of the grid's previous stage
// has counted itself done.  Stages of one grid (the sequence of ppe_project):
//   0 rho_0 = min(rho)   1 stencil constants   2 right-hand side   3 forward x
//   4 forward z          5 y solve             6 inverse z         7 inverse x
// then one refinement sweep:
//   8 residual and forward x   9 forward z   10 y solve   11 inverse z
//   12 inverse x, accumulated  13 correction and residual   14 loop test
// Further sweeps (grids whose loop test asks for one) run stages 8-14 again in
// further launches of the same kernel, inside a graph WHILE loop.
enum BatchStageKind { BS_RHO = 0, BS_CONST, BS_RHS, BS_XF, BS_ZF0, BS_Y0, BS_ZI0, BS_XI0, BS_RES, BS_ZF, BS_Y,
                      BS_ZI, BS_XA, BS_CC, BS_CHK, kBatchStages };
constexpr int kBatchThreads = 256;

struct BatchGrid {            // one grid of the batch (device copy, read-only in the kernel)
  GridDev g;
  StencilIn in;
  DevScalars* sc;
  double* f64;                // f as FP64 (may be NULL)
  df *fdf, *pdf, *upre, *vpre, *wpre;
  cpx<float>* spec;
  const cpx<float> *tw_x, *tw_z, *tw_y, *wq_y;
  const float *lam_x, *lam_y, *lam_z;
  double *out_p, *out_u, *out_v, *out_w;
  double rho0, tol, scale;    // rho0 <= 0: min(rho); scale 1 / ((nx/2) nz)
  int smax;                   // refinement sweeps at most (>= 1)
  int lpb, tkx, tky, kc;      // tiles of the x passes (radix-3 nx), z and y passes (radix-3), RHS chunk
  int stage0;                 // the grid's first stage counter (kBatchStages per grid)
};
struct BatchItem {            // tiles tile0 .. tile0 + count - 1 of one stage of one grid
  uint16_t grid;
  uint8_t stage, count;
  uint32_t tile0;
};
struct BatchCtl {
  unsigned int next;          // queue head
  int abort;                  // set on a timed-out wait: every CTA stops taking items
  int status;                 // 0, or PPE_ERR_TIMEOUT
  int err_grid, err_stage;    // the wait that ran out
  int cont_any;               // a loop test of this launch asked for another sweep
  int launches;               // launches of the kernel in the last batch run
  int pad;
};
bool batch_dims_ok(int nx, int ny, int nz);            // lengths with instances in the batched kernel
unsigned batch_stage_tiles(int nx, int ny, int nz, bool rho_given, int stage);
// tiles per queue item of a stage: about `grain` elements (cells, faces or
// spectrum values) per item, at most 255 tiles
unsigned batch_stage_chunk(int nx, int ny, int nz, int stage, long grain);
int batch_lpb(int nx);                                   // x-pass lines per tile (radix-3 nx/2)
int batch_tkx(int n, bool zpass);                        // z / y columns per tile (radix-3 lengths)
size_t batch_smem(int nx, int ny, int nz);               // dynamic shared memory of the grid's largest stage
// queue of stages [first, kBatchStages) of every grid: grids in windows of
// `window`, stage-major within a window, window w offset by w * stagger stages
// need[kBatchStages g + s]: the items of every stage (the count a waiting
// stage needs), tiles[...]: its tiles (the tile count its device function sees)
long long batch_item_count(int n, const int* nx, const int* ny, const int* nz, const int* rho_given, int first,
                           long grain);
void batch_schedule(int n, const int* nx, const int* ny, const int* nz, const int* rho_given, int window,
                    int stagger, int first, long grain, BatchItem* items, unsigned* need, unsigned* tiles);
cudaError_t batch_occupancy(size_t smem, int* ctas_per_sm);
// reset of every grid's scalars, the counters and the control block (before the first launch)
cudaError_t launch_batch_reset(const BatchGrid* grids, int ngrid, unsigned* done, int ndone, int* stop,
                               BatchCtl* ctl, cudaStream_t st);
// reset of the sweep stages' counters and the queue head (before a further sweep)
cudaError_t launch_batch_sweep_reset(const BatchGrid* grids, int ngrid, unsigned* done, BatchCtl* ctl,
                                     cudaStream_t st);
cudaError_t launch_batch(const BatchGrid* grids, int ngrid, const BatchItem* items, int nitems, unsigned* done,
                         int ndone, const unsigned* need, const unsigned* tiles, int* stop, BatchCtl* ctl,
                         unsigned long long wait_ns, int hold, int ctas, size_t smem, cudaStream_t st);
// sets the WHILE condition: another sweep if a loop test asked for one and no wait ran out
cudaError_t launch_batch_cond(BatchCtl* ctl, cudaGraphConditionalHandle h, cudaStream_t st);

// ---- launchers (k_stencil.cu) ----
// Eq. (31) divergence constraint (and the one-fluid density when rho != NULL)
cudaError_t launch_div_constraint(size_t n, const double* C, const double* comp_g, const double* comp_l,
                                  const double* mdot, const double* rho_g, const double* rho_l,
                                  const unsigned char* mask, double* S, double* rho, cudaStream_t st);
cudaError_t launch_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, cudaStream_t st,
                                double* out_p = nullptr, double* out_u = nullptr, double* out_v = nullptr,
                                double* out_w = nullptr);
cudaError_t launch_set_rho0(DevScalars* sc, double rho0, cudaStream_t st);
// Forms sc->K from sc->rho0, dt and the grid (one thread).
cudaError_t launch_make_const(const GridDev& g, DevScalars* sc, double dt, cudaStream_t st);
cudaError_t launch_rho_min(const double* rho, size_t n, DevScalars* sc, cudaStream_t st);
// u^{n+1} = u_pre - (dt/rho_0) G p with p as pairs (pdf) or FP64 (p64); also
// writes p64 from pdf when both are given.
cudaError_t launch_correct_pre(const GridDev& g, double dt, const df* upre, const df* vpre, const df* wpre,
                               const df* pdf, double* p64, const DevScalars* sc, double* u_out, double* v_out,
                               double* w_out, cudaStream_t st);
// Eq. (33) from the raw inputs (the separate ppe_correct entry point).
cudaError_t launch_correct_full(const GridDev& g, const StencilIn& in, const DevScalars* sc, double* u_out,
                                double* v_out, double* w_out, cudaStream_t st);
cudaError_t launch_df_to_d(const df* a, double* out, size_t n, cudaStream_t st);
// Eq. (33) from u_pre and p (pairs) fused with the residual r = f - L p of the
// same p into rmax[iter + 1]; outputs through sc->out_*.
cudaError_t launch_correct_check(const GridDev& g, const df* upre, const df* vpre, const df* wpre, const df* pdf,
                                 const df* fdf, DevScalars* sc, cudaStream_t st);
// Convergence test of the residual in slot sc->iter + off (off = 0: probe
// before a correction; off = 1: after correction sc->iter, from the fused
// correction kernel); sets sc->cont and, when use_handle, the WHILE condition.
cudaError_t launch_refine_check(DevScalars* sc, int smax, int off, cudaGraphConditionalHandle handle,
                                int use_handle, cudaStream_t st);

}  // namespace ppe
