// Right-hand side of the split pressure Poisson equation, Eq. (34).
//
//   f = D[beta_f G p_hat] + (rho_0/dt)(D u* - S),  beta_f = 1 - rho_0/rho_f,
//   p_hat = 2 p^n - p^{n-1}                                        (Eq. (32))
//
// Written per face as Q~_f = beta_f (p_hat_R - p_hat_L) + (rho_0/dt) h u*_f (h
// the spacing of the face's direction), so that f = sum_dir (Q~_+ - Q~_-)/h^2
// - (rho_0/dt) S.  The same face quantity also gives the explicitly
// split velocity of Eq. (33):  since 1/rho_f - 1/rho_0 = -beta_f/rho_0,
//   u^{n+1}_f = u*_f + (dt/rho_0) beta_f (G p_hat)_f - (dt/rho_0) (G p^{n+1})_f
// and this kernel stores u_pre_f = u*_f + (dt/rho_0) beta_f (G p_hat)_f, leaving
// only the pressure-gradient term for the kernel that runs after the solve.
//
// Arithmetic: FP64 inputs are split into float pairs with integer operations
// (dfloat.cuh) and every face and cell value is formed in pair arithmetic.
//
// Blocking: a CTA owns `tj` consecutive y-lines for a chunk of `kc` z-planes and
// marches upward in z.  Shared memory holds, for the current plane and the one
// above, p_hat and rho of the tj lines plus one halo line on each side (a
// 2-plane ring), and the face values Q of the x faces, y faces and the two z
// faces of the current plane.  Each input value is converted once per CTA
// (plus halo), each face is evaluated once.  f is written as float pairs (the
// forward x transform reads it back, k_xfwd) and/or as FP64.
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

struct RhsOut {
  double* f64;   // optional: f as FP64
  df* fdf;       // optional: f as pairs (kept for the residual)
  df* upre;      // optional: u_pre on x faces  [nz][ny][nx]
  df* vpre;      //           v_pre on y faces  [nz][ny+1][nx]
  df* wpre;      //           w_pre on z faces  [nz][ny][nx]
};

__global__ void __launch_bounds__(256) k_rhs_march(GridDev g, StencilIn in, DevScalars* sc, RhsOut out, int tj,
                                                   int kc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ntile = (ny + tj - 1) / tj;
  const int jt = blockIdx.x % ntile, kci = blockIdx.x / ntile;
  const int j0 = jt * tj, k0 = kci * kc;
  const int steps = min(kc, nz - k0);
  const int nl = tj + 2;  // ring lines per plane
  const int rule = in.face_rule;

  // shared layout
  df* P = reinterpret_cast<df*>(smem_raw);          // [2][nl][nx]
  df* R = P + 2 * nl * nx;                          // [2][nl][nx]
  df* QX = R + 2 * nl * nx;                         // [tj][nx]
  df* QY = QX + tj * nx;                            // [tj+1][nx]
  df* QZ = QY + (tj + 1) * nx;                      // [2][tj][nx]

  const StencilConst K = sc->K;  // formed once per call by k_make_const
  // 32-bit element offsets (grids up to 1024^3 stay below 2^32)
  const uint32_t plane = (uint32_t)ny * (uint32_t)nx;
  const uint32_t vplane = (uint32_t)(ny + 1) * (uint32_t)nx;

  // Loops below take their items in chunks of U per thread and issue all of a
  // chunk's global loads before the first use, so that a CTA waits about once
  // per phase instead of once per item.
  constexpr int UR = 6, UF = 4;
  const int nthr = blockDim.x;

  // ring slot s <- plane kk (periodic), lines j0-1 .. j0+tj
  auto load_plane = [&](int slot, int kk) {
    kk = (kk % nz + nz) % nz;
    df* Ps = P + slot * nl * nx;
    df* Rs = R + slot * nl * nx;
    const int total = nl * nx;
    for (int b0 = 0; b0 < total; b0 += UR * nthr) {
      double vn[UR], vm[UR], vr[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        const int l = (int)fdiv(idx, g.fd_nx), i = idx - l * nx;
        const int j = j0 - 1 + l;
        vn[u] = 0.0;
        vm[u] = 0.0;
        vr[u] = 1.0;
        if (idx < total && j >= 0 && j < ny) {
          const uint32_t c = (uint32_t)kk * plane + (uint32_t)(j * nx + i);
          vn[u] = __ldg(in.pn + c);
          vm[u] = __ldg(in.pnm1 + c);
          vr[u] = __ldg(in.rho + c);
        }
      }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        if (idx < total) {
          Ps[idx] = df_sub(df_ldexp2(d2df(vn[u])), d2df(vm[u]));
          Rs[idx] = d2df(vr[u]);
        }
      }
    }
  };

  // z face between plane (slot lo) and (slot hi): lines jj < tj; face index
  // kf = the upper plane's index; store Q in QZ[zs]; write w_pre if owned
  auto z_faces = [&](int slot_lo, int slot_hi, int kf, int zs, bool owned) {
    kf = (kf % nz + nz) % nz;
    const df* Pl = P + slot_lo * nl * nx;
    const df* Ph = P + slot_hi * nl * nx;
    const df* Rl = R + slot_lo * nl * nx;
    const df* Rh = R + slot_hi * nl * nx;
    const int total = tj * nx;
    for (int b0 = 0; b0 < total; b0 += UF * nthr) {
      double ws[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        const int jj = (int)fdiv(idx, g.fd_nx), i = idx - jj * nx;
        ws[u] = 0.0;
        if (idx < total && j0 + jj < ny) ws[u] = __ldg(in.w + ((uint32_t)kf * plane + (uint32_t)((j0 + jj) * nx + i)));
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        if (idx >= total) continue;
        const int jj = (int)fdiv(idx, g.fd_nx), i = idx - jj * nx;
        const int j = j0 + jj;
        df q = {0.0f, 0.0f};
        if (j < ny) {
          const int r = (jj + 1) * nx + i;
          const FaceOut fo = face_q(Rl[r], Rh[r], Pl[r], Ph[r], d2df(ws[u]), K.cz, K.gz, K, rule);
          q = fo.q;
          if (owned && out.wpre) out.wpre[(uint32_t)kf * plane + (uint32_t)(j * nx + i)] = fo.upre;
        }
        QZ[zs * tj * nx + idx] = q;
      }
    }
  };

  // prologue: plane k0-1 in slot 1, plane k0 in slot 0, face k0 -> QZ[0]
  load_plane(1, k0 - 1);
  load_plane(0, k0);
  __syncthreads();
  z_faces(1, 0, k0, 0, true);
  __syncthreads();
  load_plane(1, k0 + 1);
  __syncthreads();

  float vmax = 0.0f;
  for (int st = 0; st < steps; ++st) {
    const int k = k0 + st;
    const int a = st & 1, b = a ^ 1;  // slot of plane k, plane k+1
    const int zdn = st & 1, zup = zdn ^ 1;
    const df* Pa = P + a * nl * nx;
    const df* Ra = R + a * nl * nx;
    // ---- phase A: x faces and y faces of plane k, z face k+1
    for (int b0 = 0; b0 < tj * nx; b0 += UF * nthr) {
      double us_[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        const int jj = (int)fdiv(idx, g.fd_nx), i = idx - jj * nx;
        us_[u] = 0.0;
        if (idx < tj * nx && j0 + jj < ny) us_[u] = __ldg(in.u + ((uint32_t)k * plane + (uint32_t)((j0 + jj) * nx + i)));
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        if (idx >= tj * nx) continue;
        const int jj = (int)fdiv(idx, g.fd_nx), i = idx - jj * nx;
        const int j = j0 + jj;
        df q = {0.0f, 0.0f};
        if (j < ny) {
          const int r = (jj + 1) * nx;
          const int im = (i == 0) ? nx - 1 : i - 1;
          const FaceOut fo = face_q(Ra[r + im], Ra[r + i], Pa[r + im], Pa[r + i], d2df(us_[u]), K.cx, K.gx, K, rule);
          q = fo.q;
          if (out.upre) out.upre[(uint32_t)k * plane + (uint32_t)(j * nx + i)] = fo.upre;
        }
        QX[idx] = q;
      }
    }
    for (int b0 = 0; b0 < (tj + 1) * nx; b0 += UF * nthr) {
      double vs_[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        const int jf = (int)fdiv(idx, g.fd_nx), i = idx - jf * nx;
        vs_[u] = 0.0;
        if (idx < (tj + 1) * nx && j0 + jf <= ny) vs_[u] = __ldg(in.v + ((uint32_t)k * vplane + (uint32_t)((j0 + jf) * nx + i)));
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        if (idx >= (tj + 1) * nx) continue;
        const int jf = (int)fdiv(idx, g.fd_nx), i = idx - jf * nx;
        const int j = j0 + jf;  // face between cells j-1 and j
        df q = {0.0f, 0.0f};
        if (j <= ny) {
          const uint32_t cv = (uint32_t)k * vplane + (uint32_t)(j * nx + i);
          const df vs = d2df(vs_[u]);
          const bool own = (jf < tj) || (j == ny);
          if (j == 0 || j == ny) {
            q = df_norm(df_mulz(K.cy, vs));
            if (own && out.vpre) out.vpre[cv] = vs;
          } else {
            const int rl = jf * nx + i, rh = (jf + 1) * nx + i;
            const FaceOut fo = face_q(Ra[rl], Ra[rh], Pa[rl], Pa[rh], vs, K.cy, K.gy, K, rule);
            q = fo.q;
            if (own && out.vpre) out.vpre[cv] = fo.upre;
          }
        }
        QY[idx] = q;
      }
    }
    z_faces(a, b, k + 1, zup, k + 1 < k0 + steps);
    __syncthreads();
    // ---- phase B: cells of plane k
    for (int b0 = 0; b0 < tj * nx; b0 += UF * nthr) {
      double ss_[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        const int jj = (int)fdiv(idx, g.fd_nx), i = idx - jj * nx;
        ss_[u] = 0.0;
        if (idx < tj * nx && j0 + jj < ny) ss_[u] = __ldg(in.S + ((uint32_t)k * plane + (uint32_t)((j0 + jj) * nx + i)));
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const int idx = b0 + u * nthr + threadIdx.x;
        if (idx >= tj * nx) continue;
        const int jj = (int)fdiv(idx, g.fd_nx), i = idx - jj * nx;
        const int j = j0 + jj;
        if (j < ny) {
          const int ip = (i + 1 == nx) ? 0 : i + 1;
          // f = sum over directions of (Q~_+ - Q~_-) / h^2 - (rho_0/dt) S
          const df dxq = df_mulz(df_subz(QX[jj * nx + ip], QX[idx]), K.lx);
          const df dyq = df_mulz(df_subz(QY[(jj + 1) * nx + i], QY[idx]), K.ly);
          const df dzq = df_mulz(df_subz(QZ[zup * tj * nx + idx], QZ[zdn * tj * nx + idx]), K.lz);
          const uint32_t c = (uint32_t)k * plane + (uint32_t)(j * nx + i);
          const df f = df_norm(df_subz(df_addz(df_addz(dxq, dyq), dzq), df_mulz(K.c, d2df(ss_[u]))));
          if (out.fdf) out.fdf[c] = f;
          if (out.f64) out.f64[c] = df2d(f);
          vmax = fmaxf(vmax, fabsf(f.hi));
        }
      }
    }
    // ---- slot a (plane k) is free: load plane k+2 for the next step
    if (st + 1 < steps) load_plane(a, k + 2);
    __syncthreads();
  }
  block_max_to(&sc->fmax_bits, vmax);
}

size_t rhs_smem(int nx, int tj) {
  const size_t nl = tj + 2;
  return sizeof(df) * (4 * nl * nx + (size_t)tj * nx + (size_t)(tj + 1) * nx + 2 * (size_t)tj * nx);
}

cudaError_t launch_rhs(const GridDev& g, const StencilIn& in, DevScalars* sc, double* f64, df* fdf, df* upre,
                       df* vpre, df* wpre, int tj, int kc, cudaStream_t st) {
  RhsOut o;
  o.f64 = f64;
  o.fdf = fdf;
  o.upre = upre;
  o.vpre = vpre;
  o.wpre = wpre;
  const int ntile = (g.ny + tj - 1) / tj;
  const int nchunk = (g.nz + kc - 1) / kc;
  k_rhs_march<<<ntile * nchunk, 256, rhs_smem(g.nx, tj), st>>>(g, in, sc, o, tj, kc);
  return cudaGetLastError();
}

cudaError_t set_rhs_smem_limit() {
  return cudaFuncSetAttribute(k_rhs_march, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace ppe
