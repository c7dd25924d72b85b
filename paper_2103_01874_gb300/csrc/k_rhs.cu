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
// Arithmetic: p_hat is formed by one FP64 fused multiply-add; it and the other
// FP64 inputs are split into float pairs with integer operations (dfloat.cuh)
// and every face and cell value is formed in pair arithmetic.
//
// Blocking: a CTA owns `tj` consecutive y-lines for a chunk of `kc` z-planes and
// marches upward in z.  Each thread owns fixed (i, j) columns of the tile and
// keeps in registers the next plane's p_hat and rho and the value of the lower
// z face of its cells; shared memory holds the current plane's p_hat and rho
// (the tj lines plus one halo line on each side) and the x- and y-face values.
// Each input value is converted once per CTA (plus halo lines), each face is
// evaluated once.  f is written as float pairs (the forward x transform reads
// it back, k_xfwd) and/or as FP64.
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "pdl.cuh"
#include "stencil.cuh"
#include "rhs.cuh"

namespace ppe {

// CPT: columns per thread (tj * nx <= CPT * kRhsThreads); RULE: face density
// rule (0 arithmetic, 1 harmonic); PROJ: the projection's outputs (f as pairs
// and u_pre, v_pre, w_pre always written, f as FP64 when given) or, with
// PROJ = false, f as FP64 only (ppe_rhs)
template <int CPT, int RULE, bool PROJ>
__global__ void __launch_bounds__(kRhsThreads, (CPT <= 2) ? 3 : (CPT == 4 ? 2 : 1))
    k_rhs_march(GridDev g, StencilIn in, DevScalars* sc, RhsOut out, int tj, int kc) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ntile = (ny + tj - 1) / tj;
  const int jt = blockIdx.x % ntile, kci = blockIdx.x / ntile;
  const int j0 = jt * tj, k0 = kci * kc;
  const int steps = min(kc, nz - k0);
  const int nl = tj + 2;  // lines of the current plane held in shared memory (with halos)
  constexpr int rule = RULE;

  // shared: current plane p_hat and rho (nl lines), x-face and y-face values
  df* P = reinterpret_cast<df*>(smem_raw);  // [nl][nx]
  df* R = P + nl * nx;                      // [nl][nx]
  df* QX = R + nl * nx;                     // [tj][nx]
  df* QY = QX + tj * nx;                    // [tj+1][nx]

  const StencilConst K = sc->K;  // formed once per call by k_make_const
  // 32-bit element offsets (grids up to 1024^3 stay below 2^32)
  const uint32_t plane = (uint32_t)ny * (uint32_t)nx;
  const uint32_t vplane = (uint32_t)(ny + 1) * (uint32_t)nx;
  const int ncol = tj * nx;

  // this thread's columns (i, jj), fixed for the whole march
  int ci[CPT], cj[CPT];
  bool cv[CPT];
#pragma unroll
  for (int u = 0; u < CPT; ++u) {
    const int c = threadIdx.x + u * kRhsThreads;
    cj[u] = (int)fdiv((uint32_t)c, g.fd_nx);
    ci[u] = c - cj[u] * nx;
    cv[u] = c < ncol && j0 + cj[u] < ny;
  }
  // registers: p_hat, rho of the plane above the current one; Q of the lower z face
  df P1[CPT], R1[CPT], QZ[CPT];

  auto cell = [&](int kk, int j, int i) -> uint32_t { return (uint32_t)kk * plane + (uint32_t)(j * nx + i); };
  auto wrapk = [&](int kk) { return kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk); };  // kk in [-nz, 2 nz)

  // own columns of plane kk into (pv, rv)
  auto load_cols = [&](int kk, df* pv, df* rv) {
    kk = wrapk(kk);
    double a[CPT], b[CPT], r[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      a[u] = 0.0; b[u] = 0.0; r[u] = 1.0;
      if (cv[u]) {
        const uint32_t c = cell(kk, j0 + cj[u], ci[u]);
        a[u] = __ldg(in.pn + c);
        b[u] = __ldg(in.pnm1 + c);
        r[u] = __ldg(in.rho + c);
      }
    }
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      pv[u] = phat_of(a[u], b[u]);  // p_hat = 2 p^n - p^{n-1}
      rv[u] = d2df(r[u]);
    }
  };
  // halo lines j0-1 and j0+tj of plane kk into shared lines 0 and nl-1
  auto load_halo = [&](int kk) {
    kk = wrapk(kk);
    for (int idx = threadIdx.x; idx < 2 * nx; idx += kRhsThreads) {
      const int h = idx >= nx, i = idx - h * nx;
      const int j = h ? j0 + tj : j0 - 1;
      const int l = h ? nl - 1 : 0;
      df pv = {0.0f, 0.0f}, rv = {1.0f, 0.0f};
      if (j >= 0 && j < ny) {
        const uint32_t c = cell(kk, j, i);
        pv = phat_of(__ldg(in.pn + c), __ldg(in.pnm1 + c));
        rv = d2df(__ldg(in.rho + c));
      }
      P[l * nx + i] = pv;
      R[l * nx + i] = rv;
    }
  };
  // z face kf (between planes kf-1 and kf) of own columns from (pl, rl) below and (ph, rh) above
  auto z_face = [&](int kf, const df* pl, const df* rl, const df* ph, const df* rh, bool owned, df* q) {
    kf = wrapk(kf);
    double ws[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) ws[u] = cv[u] ? __ldg(in.w + cell(kf, j0 + cj[u], ci[u])) : 0.0;
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      q[u] = {0.0f, 0.0f};
      if (!cv[u]) continue;
      const FaceOut fo = face_q(rl[u], rh[u], pl[u], ph[u], d2df(ws[u]), K.cz, K.gz, K, rule);
      q[u] = fo.q;
      if (PROJ && owned) out.wpre[cell(kf, j0 + cj[u], ci[u])] = fo.upre;
    }
  };

  // raw next-step loads, issued a phase ahead of their use
  double us_[CPT], ss_[CPT], ws_[CPT];
  auto load_step = [&](int k) {  // u* and S of plane k, w* of face k+1, own columns
    const int kw = wrapk(k + 1);
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      us_[u] = cv[u] ? __ldg(in.u + cell(k, j0 + cj[u], ci[u])) : 0.0;
      ss_[u] = cv[u] ? __ldg(in.S + cell(k, j0 + cj[u], ci[u])) : 0.0;
      ws_[u] = cv[u] ? __ldg(in.w + cell(kw, j0 + cj[u], ci[u])) : 0.0;
    }
  };

  // prologue: plane k0 in shared memory (own lines from registers, halos
  // loaded), face k0 from planes k0-1 and k0, plane k0+1 in registers
  {
    df P0[CPT], R0[CPT];
    load_cols(k0 - 1, P1, R1);
    load_cols(k0, P0, R0);
    z_face(k0, P1, R1, P0, R0, true, QZ);
#pragma unroll
    for (int u = 0; u < CPT; ++u)
      if (threadIdx.x + u * kRhsThreads < ncol) {
        P[(cj[u] + 1) * nx + ci[u]] = P0[u];
        R[(cj[u] + 1) * nx + ci[u]] = R0[u];
      }
    load_halo(k0);
    load_cols(k0 + 1, P1, R1);
    load_step(k0);
  }
  __syncthreads();

  float vmax = 0.0f, smax = 0.0f, wmax = 0.0f;
  df wsum = {0.0f, 0.0f};  // wall flux v*(ny) - v*(0) of this CTA's wall faces
  for (int st = 0; st < steps; ++st) {
    const int k = k0 + st;
    const bool more = st + 1 < steps;
    // raw p^n, p^{n-1}, rho of plane k+2 (own columns): in flight during A and B
    double rp[CPT], rm[CPT], rr[CPT];
    if (more) {
      const int k2 = wrapk(k + 2);
#pragma unroll
      for (int u = 0; u < CPT; ++u) {
        rp[u] = 0.0; rm[u] = 0.0; rr[u] = 1.0;
        if (cv[u]) {
          const uint32_t c = cell(k2, j0 + cj[u], ci[u]);
          rp[u] = __ldg(in.pn + c);
          rm[u] = __ldg(in.pnm1 + c);
          rr[u] = __ldg(in.rho + c);
        }
      }
    }
    // ---- phase A: faces of plane k (x, y from shared; z face k+1 from registers)
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      if (threadIdx.x + u * kRhsThreads >= ncol) continue;
      df q = {0.0f, 0.0f};
      if (cv[u]) {
        const int r = (cj[u] + 1) * nx;
        const int i = ci[u], im = (i == 0) ? nx - 1 : i - 1;
        const FaceOut fo = face_q(R[r + im], R[r + i], P[r + im], P[r + i], d2df(us_[u]), K.cx, K.gx, K, rule);
        q = fo.q;
        if (PROJ) out.upre[cell(k, j0 + cj[u], i)] = fo.upre;
      }
      QX[cj[u] * nx + ci[u]] = q;
    }
    {
      constexpr int UY = 4;
      const int ny_faces = (tj + 1) * nx;
      for (int b0 = 0; b0 < ny_faces; b0 += UY * kRhsThreads) {
        double vv[UY];
#pragma unroll
        for (int u = 0; u < UY; ++u) {
          const int idx = b0 + u * kRhsThreads + threadIdx.x;
          const int jf = (int)fdiv((uint32_t)idx, g.fd_nx), i = idx - jf * nx;
          vv[u] = (idx < ny_faces && j0 + jf <= ny)
                      ? __ldg(in.v + ((uint32_t)k * vplane + (uint32_t)((j0 + jf) * nx + i))) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < UY; ++u) {
          const int idx = b0 + u * kRhsThreads + threadIdx.x;
          if (idx >= ny_faces) continue;
          const int jf = (int)fdiv((uint32_t)idx, g.fd_nx), i = idx - jf * nx;
          const int j = j0 + jf;  // face between cells j-1 and j
          df q = {0.0f, 0.0f};
          if (j <= ny) {
            const uint32_t cvv = (uint32_t)k * vplane + (uint32_t)(j * nx + i);
            const df vs = d2df(vv[u]);
            const bool own = (jf < tj) || (j == ny);
            if (j == ny && g.top_open) {  // open top: p = 0 on the face, ghost -p_hat above
              const int rl = jf * nx + i;
              const FaceOut fo = face_q(R[rl], R[rl], P[rl], df_neg(P[rl]), vs, K.cy, K.gy, K, rule);
              q = fo.q;
              if (PROJ && own) out.vpre[cvv] = fo.upre;
            } else if (j == 0 || j == ny) {  // wall
              q = df_norm(df_mulz(K.cy, vs));
              if (PROJ && own) out.vpre[cvv] = vs;
              wsum = (j == ny) ? df_addz(wsum, vs) : df_subz(wsum, vs);
              wmax = fmaxf(wmax, fabsf(vs.hi));
            } else {
              const int rl = jf * nx + i, rh = (jf + 1) * nx + i;
              const FaceOut fo = face_q(R[rl], R[rh], P[rl], P[rh], vs, K.cy, K.gy, K, rule);
              q = fo.q;
              if (PROJ && own) out.vpre[cvv] = fo.upre;
            }
          }
          QY[idx] = q;
        }
      }
    }
    df QZup[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      QZup[u] = {0.0f, 0.0f};
      if (!cv[u]) continue;
      const int r = (cj[u] + 1) * nx + ci[u];
      const FaceOut fo = face_q(R[r], R1[u], P[r], P1[u], d2df(ws_[u]), K.cz, K.gz, K, rule);
      QZup[u] = fo.q;
      if (PROJ && k + 1 < k0 + steps) out.wpre[cell(wrapk(k + 1), j0 + cj[u], ci[u])] = fo.upre;
    }
    __syncthreads();
    // ---- phase B: cells of plane k
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      if (!cv[u]) continue;
      const int i = ci[u], jj = cj[u];
      const int ip = (i + 1 == nx) ? 0 : i + 1;
      // f = sum over directions of (Q~_+ - Q~_-) / h^2 - (rho_0/dt) S
      const df dxq = df_mulz(df_subz(QX[jj * nx + ip], QX[jj * nx + i]), K.lx);
      const df dyq = df_mulz(df_subz(QY[(jj + 1) * nx + i], QY[jj * nx + i]), K.ly);
      const df dzq = df_mulz(df_subz(QZup[u], QZ[u]), K.lz);
      const uint32_t c = cell(k, j0 + jj, i);
      const df sv = d2df(ss_[u]);
      const df f = df_norm(df_subz(df_addz(df_addz(dxq, dyq), dzq), df_mulz(K.c, sv)));
      smax = fmaxf(smax, fabsf(sv.hi));
      if (PROJ) out.fdf[c] = f;
      if (!PROJ || out.f64) out.f64[c] = df2d(f);
      vmax = fmaxf(vmax, fabsf(f.hi));
      QZ[u] = QZup[u];
    }
    if (more) {
      load_step(k + 1);  // next step's u*, S, w*: in flight during the rest of this step
      __syncthreads();
      // ---- phase C: plane k+1 becomes current; plane k+2 (loaded above) into registers
#pragma unroll
      for (int u = 0; u < CPT; ++u)
        if (threadIdx.x + u * kRhsThreads < ncol) {
          P[(cj[u] + 1) * nx + ci[u]] = P1[u];
          R[(cj[u] + 1) * nx + ci[u]] = R1[u];
        }
      load_halo(k + 1);
#pragma unroll
      for (int u = 0; u < CPT; ++u) {
        P1[u] = phat_of(rp[u], rm[u]);
        R1[u] = d2df(rr[u]);
      }
      __syncthreads();
    }
  }
  block_max_to(&sc->fmax_bits, vmax);
  block_max_to(&sc->smax_bits, smax);
  block_max_to(&sc->wallv_bits, wmax);
  // wall tiles: the CTA's wall flux, totalled in a fixed order by a later
  // kernel (finish_sums), so no grid-wide fence here
  if (j0 == 0 || j0 + tj >= ny) block_pair_sums(wsum, df{0.0f, 0.0f}, sc->part + blockIdx.x);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rhs_tiles = ntile;
    sc->rhs_chunks = (nz + kc - 1) / kc;
  }
}

__global__ void k_finish_sums(GridDev g, DevScalars* sc) { finish_sums(sc, g); }

// Column-stack form of the march (rhs.cuh): one CTA per tile.
template <int S, int RULE, bool PROJ>
__global__ void __launch_bounds__(kRhsThreads, (S <= 2) ? 3 : (S == 4 ? 2 : 1))
    k_rhs_stack(GridDev g, StencilIn in, DevScalars* sc, RhsOut out, int kc) {
  pdl_enter();
  rhs_stack_tile<S, RULE, PROJ>(g, in, sc, out, kc, blockIdx.x);
}

// Lines per tile: the stack form (nx <= 256) has 256 / nx stacks of `lines`
// lines each; the general form has `lines` lines.
int rhs_tile_lines(int nx, int lines) { return nx <= kRhsThreads ? (kRhsThreads / nx) * lines : lines; }

size_t rhs_smem(int nx, int lines) {
  const size_t tj = rhs_tile_lines(nx, lines), nl = tj + 2;
  if (nx <= kRhsThreads) return sizeof(df) * (2 * nl * nx + tj * nx);
  return sizeof(df) * (2 * nl * nx + tj * nx + (tj + 1) * nx);
}

int rhs_max_lines(int nx) {
  if (nx <= kRhsThreads) return kRhsMaxCols;
  int tj = 8;
  while (tj > 1 && tj * nx > kRhsThreads * kRhsMaxCols) tj /= 2;
  return tj;
}

cudaError_t launch_rhs(const GridDev& g, const StencilIn& in, DevScalars* sc, double* f64, df* fdf, df* upre,
                       df* vpre, df* wpre, int tj, int kc, cudaStream_t st) {
  RhsOut o;
  o.f64 = f64;
  o.fdf = fdf;
  o.upre = upre;
  o.vpre = vpre;
  o.wpre = wpre;
  const int tile = rhs_tile_lines(g.nx, tj);
  const int ntile = (g.ny + tile - 1) / tile;
  const int nchunk = (g.nz + kc - 1) / kc;
  const size_t sm = rhs_smem(g.nx, tj);
  const int grid = ntile * nchunk;
  const bool proj = fdf != nullptr;
  if (proj && !(upre && vpre && wpre)) return cudaErrorInvalidValue;
  if (!proj && !f64) return cudaErrorInvalidValue;
  if (g.nx <= kRhsThreads) {
    // column-stack form: tj is the stack height S
    auto go = [&](auto kernel) { launch_pdl(kernel, grid, kRhsThreads, sm, st, g, in, sc, o, kc); };
#define PPE_STACK_CASE(C)                                                        \
    if (tj == C) {                                                               \
      if (in.face_rule == 0) {                                                   \
        if (proj) go(k_rhs_stack<C, 0, true>); else go(k_rhs_stack<C, 0, false>); \
      } else {                                                                   \
        if (proj) go(k_rhs_stack<C, 1, true>); else go(k_rhs_stack<C, 1, false>); \
      }                                                                          \
    }
    PPE_STACK_CASE(1)
    PPE_STACK_CASE(2)
    PPE_STACK_CASE(4)
    PPE_STACK_CASE(8)
#undef PPE_STACK_CASE
    return cudaGetLastError();
  }
  const int ncol = tj * g.nx;
  const int cpt = ncol <= kRhsThreads ? 1 : ncol <= 2 * kRhsThreads ? 2 : ncol <= 4 * kRhsThreads ? 4 : 8;
  auto go = [&](auto kernel) { launch_pdl(kernel, grid, kRhsThreads, sm, st, g, in, sc, o, tj, kc); };
  // instance table: [cpt][rule][proj]
#define PPE_RHS_CASE(C)                                                        \
  if (cpt == C) {                                                              \
    if (in.face_rule == 0) {                                                   \
      if (proj) go(k_rhs_march<C, 0, true>); else go(k_rhs_march<C, 0, false>); \
    } else {                                                                   \
      if (proj) go(k_rhs_march<C, 1, true>); else go(k_rhs_march<C, 1, false>); \
    }                                                                          \
  }
  PPE_RHS_CASE(1)
  PPE_RHS_CASE(2)
  PPE_RHS_CASE(4)
  PPE_RHS_CASE(8)
#undef PPE_RHS_CASE
  return cudaGetLastError();
}

namespace {
// Opt-in dynamic shared memory of one instance: the per-CTA maximum minus the
// instance's static shared memory (the reduction scratch).
template <typename K>
cudaError_t raise_smem(K kernel, size_t* dyn_max) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  const size_t cap = kSmemPerCta - a.sharedSizeBytes;
  if (dyn_max && cap < *dyn_max) *dyn_max = cap;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}
}  // namespace

cudaError_t launch_finish_sums(const GridDev& g, DevScalars* sc, cudaStream_t st) {
  k_finish_sums<<<1, 256, 0, st>>>(g, sc);
  return cudaGetLastError();
}

template <int C>
cudaError_t raise_rhs(size_t* cap) {
  cudaError_t e = raise_smem(k_rhs_march<C, 0, true>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_march<C, 0, false>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_march<C, 1, true>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_march<C, 1, false>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_stack<C, 0, true>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_stack<C, 0, false>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_stack<C, 1, true>, cap);
  if (e == cudaSuccess) e = raise_smem(k_rhs_stack<C, 1, false>, cap);
  return e;
}

cudaError_t set_rhs_smem_limit() {
  size_t cap = kSmemPerCta;
  cudaError_t e = raise_rhs<1>(&cap);
  if (e == cudaSuccess) e = raise_rhs<2>(&cap);
  if (e == cudaSuccess) e = raise_rhs<4>(&cap);
  if (e == cudaSuccess) e = raise_rhs<8>(&cap);
  return e;
}

size_t rhs_smem_limit() {
  size_t cap = kSmemPerCta;
  if (raise_rhs<1>(&cap) != cudaSuccess || raise_rhs<2>(&cap) != cudaSuccess || raise_rhs<4>(&cap) != cudaSuccess ||
      raise_rhs<8>(&cap) != cudaSuccess)
    return 0;
  return cap;
}

}  // namespace ppe
