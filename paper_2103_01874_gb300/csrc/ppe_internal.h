// Internal declarations shared by the libppe translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fft.cuh"

namespace ppe {

constexpr int kMaxSweeps = 16;
constexpr int kMaxDim = 1024;

// Device-resident scalars of one plan.  Non-negative doubles are kept as their
// IEEE bit patterns so that atomicMax / atomicMin on unsigned 64-bit integers
// order them correctly.
struct DevScalars {
  unsigned long long rho0_bits;                 // rho_0 (min(rho) or the given value)
  unsigned long long fmax_bits;                 // ||f||_inf
  unsigned long long rmax_bits[kMaxSweeps + 2]; // ||f - L p||_inf measured before sweep s
  int done;                                     // refinement converged
  int last_slot;                                // slot of the last residual checked (-1: none)
  int sweeps;                                   // sweeps run
  double tol;                                   // refinement tolerance (relative)
};

struct GridDev {
  int nx, ny, nz;
  double idx, idy, idz;  // 1/dx, 1/dy, 1/dz
};

// Inputs of the right-hand side (Eq. (34)) and of the correction (Eq. (33)).
struct StencilIn {
  const double *u, *v, *w, *S, *rho, *pn, *pnm1;
  const double* f;   // SRC_F / SRC_RESID: the right-hand side
  const double* p;   // SRC_RESID / correction: the pressure
  double inv_dt;
  double dt;
  int face_rule;     // 0 arithmetic, 1 harmonic
};

enum XSource { SRC_RHS = 0, SRC_F = 1, SRC_RESID = 2 };

// ---- launchers (k_spectral.cu) ----
template <typename T>
cudaError_t launch_xfwd(int src, bool do_fft, const GridDev& g, const StencilIn& in, DevScalars* sc,
                        int sweep_slot, double* f_out, cpx<T>* spec, const RadixPlan& rp_half,
                        const cpx<T>* tw_x, int lpb, cudaStream_t st);
template <typename T>
cudaError_t launch_zfft(bool inverse, const GridDev& g, cpx<T>* spec, const RadixPlan& rp,
                        const cpx<T>* tw_z, int tkx, const DevScalars* sc, cudaStream_t st);
template <typename T>
cudaError_t launch_ythomas(const GridDev& g, cpx<T>* spec, const T* tab, const int* line_off,
                           const int* line_len, T a, const DevScalars* sc, cudaStream_t st);
template <typename T>
cudaError_t launch_xinv(bool accumulate, const GridDev& g, const cpx<T>* spec, double* p, double scale,
                        const RadixPlan& rp_half, const cpx<T>* tw_x, int lpb, const DevScalars* sc,
                        cudaStream_t st);
template <typename T>
size_t xfwd_smem(int nx, int lpb);
template <typename T>
size_t zfft_smem(int nz, int tkx);
template <typename T>
size_t xinv_smem(int nx, int lpb);
template <typename T>
cudaError_t set_smem_limits();

// ---- launchers (k_stencil.cu) ----
cudaError_t launch_init_scalars(DevScalars* sc, double rho0, double tol, int keep_rho0, cudaStream_t st);
cudaError_t launch_set_rho0(DevScalars* sc, double rho0, cudaStream_t st);
cudaError_t launch_rho_min(const double* rho, size_t n, DevScalars* sc, cudaStream_t st);
cudaError_t launch_correct(const GridDev& g, const StencilIn& in, const DevScalars* sc, double* u_out,
                           double* v_out, double* w_out, cudaStream_t st);
cudaError_t launch_refine_check(DevScalars* sc, int sweep, int smax, cudaStream_t st);

}  // namespace ppe
