// Column-stack form of the right-hand side of Eq. (34) as a device function
// of the tile index, shared by its own kernel (k_rhs.cu) and the persistent
// batched kernel (k_batch.cu).  The arithmetic is described in k_rhs.cu.
#pragma once
#include "dfloat.cuh"
#include "ppe_internal.h"
#include "stencil.cuh"

namespace ppe {

constexpr int kRhsThreads = 256;
constexpr int kRhsMaxCols = 8;  // columns per thread: tj * nx <= 2048

struct RhsOut {
  double* f64;   // optional: f as FP64
  df* fdf;       // optional: f as pairs (kept for the residual)
  df* upre;      // optional: u_pre on x faces  [nz][ny][nx]
  df* vpre;      //           v_pre on y faces  [nz][ny+1][nx]
  df* wpre;      //           w_pre on z faces  [nz][ny][nx]
};

// Column-stack form of the march for nx <= 256 (the same face and cell
// arithmetic as k_rhs_march, bit for bit).  The CTA's 256 threads form
// nstk = 256 / nx stacks; thread (s, i) owns x position i of the S consecutive
// lines s*S .. s*S + S - 1 of the tile (tile height nstk * S lines).  The own
// lines' p_hat and rho of the current plane stay in registers, so the thread
// evaluates the y faces below, between and above its lines from registers
// (only the line below and the line above its stack come from shared memory,
// as do the x neighbours), and the y-face values never go through shared
// memory; the x faces are exchanged through shared memory for the cell
// divergence.  Faces between two stacks are evaluated by both (same bits).
// INT: the tile and its halo lines lie strictly inside the walls (no wall or
// open-top face, every line in range), so the boundary branches drop out.
template <int S, int RULE, bool PROJ, bool INT>
__device__ __forceinline__ void rhs_stack_body(const GridDev& g, const StencilIn& in, DevScalars* sc,
                                               const RhsOut& out, int kc, uint32_t bid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nstk = kRhsThreads / nx;
  const int tj = nstk * S;  // lines per tile
  const int ntile = (ny + tj - 1) / tj;
  const int jt = (int)(bid % ntile), kci = (int)(bid / ntile);
  const int j0 = jt * tj, k0 = kci * kc;
  const int steps = min(kc, nz - k0);
  const int nl = tj + 2;
  constexpr int rule = RULE;

  df* P = reinterpret_cast<df*>(smem_raw);  // [nl][nx]: row r holds tile line r - 1
  df* R = P + nl * nx;                      // [nl][nx]
  df* QX = R + nl * nx;                     // [tj][nx]

  const StencilConst K = sc->K;
  const uint32_t plane = (uint32_t)ny * (uint32_t)nx;
  const uint32_t vplane = (uint32_t)(ny + 1) * (uint32_t)nx;

  const int stk = (int)fdiv((uint32_t)threadIdx.x, g.fd_nx);
  const int i = (int)threadIdx.x - stk * nx;
  const bool active = stk < nstk;
  const int jb = stk * S;                    // first own line (tile coordinates)
  const int im = (i == 0) ? nx - 1 : i - 1;
  const int ip = (i + 1 == nx) ? 0 : i + 1;
  bool cv[S];
#pragma unroll
  for (int l = 0; l < S; ++l) cv[l] = active && (INT || j0 + jb + l < ny);

  auto cell = [&](int kk, int j) -> uint32_t { return (uint32_t)kk * plane + (uint32_t)(j * nx + i); };
  uint32_t coff[S];  // offsets of the own lines within a plane
#pragma unroll
  for (int l = 0; l < S; ++l) coff[l] = (uint32_t)((j0 + jb + l) * nx + i);
  auto cellL = [&](int kk, int l) -> uint32_t { return (uint32_t)kk * plane + coff[l]; };
  auto wrapk = [&](int kk) { return kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk); };  // kk in [-nz, 2 nz)

  // own lines of plane kk
  auto load_cols = [&](int kk, df* pv, df* rv) {
    kk = wrapk(kk);
    double a[S], b[S], r[S];
#pragma unroll
    for (int l = 0; l < S; ++l) {
      a[l] = 0.0; b[l] = 0.0; r[l] = 1.0;
      if (cv[l]) {
        const uint32_t c = cellL(kk, l);
        a[l] = __ldg(in.pn + c);
        b[l] = __ldg(in.pnm1 + c);
        r[l] = __ldg(in.rho + c);
      }
    }
#pragma unroll
    for (int l = 0; l < S; ++l) {
      pv[l] = phat_of(a[l], b[l]);  // p_hat = 2 p^n - p^{n-1}
      rv[l] = d2df(r[l]);
    }
  };
  // halo lines j0-1 and j0+tj of plane kk into shared rows 0 and nl-1
  auto load_halo = [&](int kk) {
    kk = wrapk(kk);
    for (int idx = threadIdx.x; idx < 2 * nx; idx += kRhsThreads) {
      const int h = idx >= nx, x = idx - h * nx;
      const int j = h ? j0 + tj : j0 - 1;
      const int row = h ? nl - 1 : 0;
      df pv = {0.0f, 0.0f}, rv = {1.0f, 0.0f};
      if (INT || (j >= 0 && j < ny)) {
        const uint32_t c = (uint32_t)kk * plane + (uint32_t)(j * nx + x);
        pv = phat_of(__ldg(in.pn + c), __ldg(in.pnm1 + c));
        rv = d2df(__ldg(in.rho + c));
      }
      P[row * nx + x] = pv;
      R[row * nx + x] = rv;
    }
  };
  auto store_rows = [&](const df* pv, const df* rv) {
    if (!active) return;
#pragma unroll
    for (int l = 0; l < S; ++l) {
      P[(jb + l + 1) * nx + i] = pv[l];
      R[(jb + l + 1) * nx + i] = rv[l];
    }
  };

  // raw next-step loads, issued a phase ahead of their use: u*, S of plane k,
  // w* of face k+1 (own lines), v* of the y faces jb .. jb+S of plane k
  double us_[S], ss_[S], ws_[S], vs_[S + 1];
  auto load_step = [&](int k) {
    const int kw = wrapk(k + 1);
#pragma unroll
    for (int l = 0; l < S; ++l) {
      us_[l] = cv[l] ? __ldg(in.u + cellL(k, l)) : 0.0;
      ss_[l] = cv[l] ? __ldg(in.S + cellL(k, l)) : 0.0;
      ws_[l] = cv[l] ? __ldg(in.w + cellL(kw, l)) : 0.0;
    }
#pragma unroll
    for (int f = 0; f <= S; ++f) {
      const int j = j0 + jb + f;
      vs_[f] = (active && (INT || j <= ny)) ? __ldg(in.v + ((uint32_t)k * vplane + (uint32_t)(j * nx + i))) : 0.0;
    }
  };

  df PC[S], RC[S], P1[S], R1[S], QZ[S];
  // prologue: plane k0 current (registers and shared rows), face k0, plane k0+1 in registers
  {
    df Pm[S], Rm[S];
    load_cols(k0 - 1, Pm, Rm);
    load_cols(k0, PC, RC);
    {
      const int kf = wrapk(k0);
      double w0[S];
#pragma unroll
      for (int l = 0; l < S; ++l) w0[l] = cv[l] ? __ldg(in.w + cellL(kf, l)) : 0.0;
#pragma unroll
      for (int l = 0; l < S; ++l) {
        QZ[l] = {0.0f, 0.0f};
        if (!cv[l]) continue;
        const FaceOut fo = face_q(Rm[l], RC[l], Pm[l], PC[l], d2df(w0[l]), K.cz, K.gz, K, rule);
        QZ[l] = fo.q;
        if (PROJ) out.wpre[cellL(kf, l)] = fo.upre;
      }
    }
    store_rows(PC, RC);
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
    double rp[S], rm[S], rr[S];
    if (more) {
      const int k2 = wrapk(k + 2);
#pragma unroll
      for (int l = 0; l < S; ++l) {
        rp[l] = 0.0; rm[l] = 0.0; rr[l] = 1.0;
        if (cv[l]) {
          const uint32_t c = cellL(k2, l);
          rp[l] = __ldg(in.pn + c);
          rm[l] = __ldg(in.pnm1 + c);
          rr[l] = __ldg(in.rho + c);
        }
      }
    }
    // ---- phase A: x faces (shared x neighbour), y faces and the upper z face (registers)
    df QXo[S], QY[S + 1], QZup[S];
#pragma unroll
    for (int l = 0; l < S; ++l) {
      QXo[l] = {0.0f, 0.0f};
      if (!cv[l]) continue;
      const int r = (jb + l + 1) * nx;
      const FaceOut fo = face_q(R[r + im], RC[l], P[r + im], PC[l], d2df(us_[l]), K.cx, K.gx, K, rule);
      QXo[l] = fo.q;
      if (PROJ) out.upre[cellL(k, l)] = fo.upre;
    }
    if (active) {
#pragma unroll
      for (int l = 0; l < S; ++l) QX[(jb + l) * nx + i] = QXo[l];
    }
#pragma unroll
    for (int f = 0; f <= S; ++f) {  // face between tile lines jb+f-1 and jb+f
      QY[f] = {0.0f, 0.0f};
      const int j = j0 + jb + f;
      if (!active || (!INT && j > ny)) continue;
      const df vs = d2df(vs_[f]);
      const uint32_t cvv = (uint32_t)k * vplane + (uint32_t)(j * nx + i);
      // a face belongs to the stack holding the line above it; the top wall to
      // the stack holding line ny - 1
      const bool own = INT ? (f < S) : ((f < S && j < ny) || (j == ny && f >= 1));
      if (!INT && j == ny && g.top_open) {  // open top: p = 0 on the face, ghost -p_hat above
        const df rl = (f == 0) ? R[(jb) * nx + i] : RC[f > 0 ? f - 1 : 0];
        const df pl = (f == 0) ? P[(jb) * nx + i] : PC[f > 0 ? f - 1 : 0];
        const FaceOut fo = face_q(rl, rl, pl, df_neg(pl), vs, K.cy, K.gy, K, rule);
        QY[f] = fo.q;
        if (PROJ && own) out.vpre[cvv] = fo.upre;
      } else if (!INT && (j == 0 || j == ny)) {  // wall
        QY[f] = df_norm(df_mulz(K.cy, vs));
        if (PROJ && own) out.vpre[cvv] = vs;
        if (own) {
          wsum = (j == ny) ? df_addz(wsum, vs) : df_subz(wsum, vs);
          wmax = fmaxf(wmax, fabsf(vs.hi));
        }
      } else {
        const df rl = (f == 0) ? R[(jb) * nx + i] : RC[f > 0 ? f - 1 : 0];
        const df pl = (f == 0) ? P[(jb) * nx + i] : PC[f > 0 ? f - 1 : 0];
        const df rh = (f == S) ? R[(jb + S + 1) * nx + i] : RC[f < S ? f : 0];
        const df ph = (f == S) ? P[(jb + S + 1) * nx + i] : PC[f < S ? f : 0];
        const FaceOut fo = face_q(rl, rh, pl, ph, vs, K.cy, K.gy, K, rule);
        QY[f] = fo.q;
        if (PROJ && own) out.vpre[cvv] = fo.upre;
      }
    }
#pragma unroll
    for (int l = 0; l < S; ++l) {
      QZup[l] = {0.0f, 0.0f};
      if (!cv[l]) continue;
      const FaceOut fo = face_q(RC[l], R1[l], PC[l], P1[l], d2df(ws_[l]), K.cz, K.gz, K, rule);
      QZup[l] = fo.q;
      if (PROJ && k + 1 < k0 + steps) out.wpre[cellL(wrapk(k + 1), l)] = fo.upre;
    }
    __syncthreads();
    // ---- phase B: cells of plane k
#pragma unroll
    for (int l = 0; l < S; ++l) {
      if (!cv[l]) continue;
      // f = sum over directions of (Q~_+ - Q~_-) / h^2 - (rho_0/dt) S
      const df dxq = df_mulz(df_subz(QX[(jb + l) * nx + ip], QXo[l]), K.lx);
      const df dyq = df_mulz(df_subz(QY[l + 1], QY[l]), K.ly);
      const df dzq = df_mulz(df_subz(QZup[l], QZ[l]), K.lz);
      const uint32_t c = cellL(k, l);
      const df sv = d2df(ss_[l]);
      const df f = df_norm(df_subz(df_addz(df_addz(dxq, dyq), dzq), df_mulz(K.c, sv)));
      smax = fmaxf(smax, fabsf(sv.hi));
      if (PROJ) out.fdf[c] = f;
      if (!PROJ || out.f64) out.f64[c] = df2d(f);
      vmax = fmaxf(vmax, fabsf(f.hi));
      QZ[l] = QZup[l];
    }
    if (more) {
      load_step(k + 1);
      // ---- phase C: plane k+1 becomes current; plane k+2 (loaded above) into
      // registers.  Phase B reads only QX, so the rows can be rewritten without
      // a barrier; the barrier below orders them before the next phase A.
#pragma unroll
      for (int l = 0; l < S; ++l) {
        PC[l] = P1[l];
        RC[l] = R1[l];
      }
      store_rows(PC, RC);
      load_halo(k + 1);
#pragma unroll
      for (int l = 0; l < S; ++l) {
        P1[l] = phat_of(rp[l], rm[l]);
        R1[l] = d2df(rr[l]);
      }
      __syncthreads();
    }
  }
  block_max_to(&sc->fmax_bits, vmax);
  block_max_to(&sc->smax_bits, smax);
  block_max_to(&sc->wallv_bits, wmax);
  if (j0 == 0 || j0 + tj >= ny) block_pair_sums(wsum, df{0.0f, 0.0f}, sc->part + bid);
  if (bid == 0 && threadIdx.x == 0) {
    sc->rhs_tiles = ntile;
    sc->rhs_chunks = (nz + kc - 1) / kc;
  }
}

// One tile (CTA index bid) of the column-stack march: the interior form when
// the tile and its halo lines lie strictly inside the walls.
template <int S, int RULE, bool PROJ>
__device__ __forceinline__ void rhs_stack_tile(const GridDev& g, const StencilIn& in, DevScalars* sc,
                                               const RhsOut& out, int kc, uint32_t bid) {
  const int tj = (kRhsThreads / g.nx) * S;
  const int ntile = (g.ny + tj - 1) / tj;
  const int j0 = (int)(bid % ntile) * tj;
  if (j0 > 0 && j0 + tj < g.ny)  // uniform over the CTA
    rhs_stack_body<S, RULE, PROJ, true>(g, in, sc, out, kc, bid);
  else
    rhs_stack_body<S, RULE, PROJ, false>(g, in, sc, out, kc, bid);
}

}  // namespace ppe
