// y pass of the FP32 solve with walls as a tridiagonal solve in scan form.
#include "ppe_internal.h"

namespace ppe {

namespace {

// y pass of the FP32 solve with walls as the tridiagonal (Thomas) solve of
// k_ythomas, written as two affine scans so that a line is shared by 16
// threads.  Per (kx, kz) line the forward elimination is the recurrence
// xt_j = (d_j - a xt_{j-1}) m_j = alpha_j xt_{j-1} + beta_j (alpha_j = -a m_j,
// beta_j = d_j m_j) and the back substitution x_j = xt_j - a m_j x_{j+1}; both
// are compositions of affine maps.  Thread (c, t) of a CTA owns column kx0 + c
// (16 consecutive kx: a warp's loads are two 128-byte rows) and the S
// consecutive j of segment t (16 segments); it composes its segment's maps,
// the segments' maps are combined in order through shared memory, and each
// thread replays its segment from its incoming value.  Every element is read
// once and written once; nothing else crosses shared memory.
// The singular line kx = kz = 0 of the walls (the 1-D Neumann Laplacian, whose
// elimination in FP32 would lose the digits the refinement needs) is solved in
// FP64 from its flux form: with q_j = a (x_{j+1} - x_j), q_j - q_{j-1} = d_j -
// mean(d) (q_{-1} = 0), so q and then a x are two prefix sums (the CTA's
// threads, in shared memory); x is then shifted to the mean zmode (the value
// that keeps p zero-mean, as the cosine-transform y pass sets the zero mode).
// Inclusive prefix sums of v[0 .. n) in place (n <= 2 blockDim.x; Hillis-Steele
// steps, every thread of the CTA calling).
__device__ __forceinline__ void block_scan2(double* vx, double* vy, int n) {
  for (int o = 1; o < n; o *= 2) {
    double ax[2], ay[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = threadIdx.x + h * blockDim.x;
      ax[h] = (j < n && j >= o) ? vx[j - o] : 0.0;
      ay[h] = (j < n && j >= o) ? vy[j - o] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = threadIdx.x + h * blockDim.x;
      if (j < n) {
        vx[j] += ax[h];
        vy[j] += ay[h];
      }
    }
    __syncthreads();
  }
}

// The singular line kx = kz = 0 (the 1-D Neumann Laplacian) in FP64 by the
// whole CTA: with q_j = a (x_{j+1} - x_j), q_j = sum over i <= j of (d_i -
// mean d), a x_j = sum over i < j of q_i (x_0 = 0); then x takes the mean zm.
// The solution goes to out[0 .. ny).
__device__ __noinline__ void singular_line(const cpx<float>* col, int ny, int nxh, double a, double zm,
                                           cpx<float>* out, double* vx, double* vy) {
  const int n = ny;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const cpx<float> v = col[(size_t)j * nxh];
    vx[j] = (double)v.x;
    vy[j] = (double)v.y;
  }
  __syncthreads();
  block_scan2(vx, vy, n);  // prefix sums of d
  const double mdx = vx[n - 1] / n, mdy = vy[n - 1] / n;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {  // q_j
    vx[j] -= (j + 1) * mdx;
    vy[j] -= (j + 1) * mdy;
  }
  __syncthreads();
  double qx[2], qy[2];
  for (int h = 0; h < 2; ++h) {
    const int j = threadIdx.x + h * blockDim.x;
    qx[h] = j < n ? vx[j] : 0.0;
    qy[h] = j < n ? vy[j] : 0.0;
  }
  block_scan2(vx, vy, n);  // sums of q up to j
  for (int h = 0; h < 2; ++h) {  // a x_j: the sum below j
    const int j = threadIdx.x + h * blockDim.x;
    if (j < n) {
      qx[h] = vx[j] - qx[h];
      qy[h] = vy[j] - qy[h];
    }
  }
  __syncthreads();
  for (int h = 0; h < 2; ++h) {
    const int j = threadIdx.x + h * blockDim.x;
    if (j < n) {
      vx[j] = qx[h];
      vy[j] = qy[h];
    }
  }
  __syncthreads();
  block_scan2(vx, vy, n);  // the total of a x
  const double cx = vx[n - 1] / n, cy = vy[n - 1] / n, ia = 1.0 / a;
  for (int h = 0; h < 2; ++h) {
    const int j = threadIdx.x + h * blockDim.x;
    if (j < n) out[j] = {(float)((qx[h] - cx) * ia + zm), (float)((qy[h] - cy) * ia)};
  }
  __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(256, (S <= 4 ? 4 : (S == 8 ? 3 : (S == 16 ? 2 : 1)))) k_ythomas_scan(GridDev g, cpx<float>* spec, const float* __restrict__ tab,
                                                      const int* __restrict__ line_off,
                                                      const int* __restrict__ line_len, float a,
                                                      const DevScalars* zsc) {
  constexpr int L = 16, T = 16;
  __shared__ float sA[T][L];
  __shared__ cpx<float> sB[T][L];
  __shared__ cpx<float> sline[16 * S];       // the singular line's solution (CTA kz = 0, kx0 = 0)
  __shared__ double sx[16 * S], sy[16 * S];  // its FP64 scans
  const int nxh = g.nx / 2 + 1, ny = g.ny;
  const int ntile = (nxh + L - 1) / L;
  const int kz = blockIdx.x / ntile, kx0 = (blockIdx.x - kz * ntile) * L;
  const int c = threadIdx.x & (L - 1), t = threadIdx.x / L;
  const int kx = kx0 + c;
  const bool valid = kx < nxh;
  const int j0 = t * S;
  cpx<float>* col = spec + (size_t)kz * ny * nxh + kx;
  const bool singular = kz == 0 && kx == 0;  // (column 0 of the CTA kz = 0, kx0 = 0)
  const bool sing_cta = kz == 0 && kx0 == 0;  // uniform over the CTA
  if (sing_cta) singular_line(spec, ny, nxh, (double)a, zsc ? zsc->zmode : 0.0, sline, sx, sy);  // (kz = kx = 0)
  int off = 0, J = 0;
  float m_inf = 0.0f, m_last = 0.0f;
  if (valid) {
    const int line = kz * nxh + kx;
    off = line_off[line];
    J = line_len[line];
    m_inf = tab[off];
    m_last = tab[off + 1];
  }
  cpx<float> d[S];
  float m[S];
#pragma unroll
  for (int u = 0; u < S; ++u) {
    const int jj = j0 + u;
    d[u] = {0.0f, 0.0f};
    m[u] = 0.0f;
    if (valid && jj < ny) {
      d[u] = col[(size_t)jj * nxh];
      m[u] = jj < J ? tab[off + 2 + jj] : (jj < ny - 1 ? m_inf : m_last);
    }
  }
  // forward elimination: this segment's map xt_out = A xt_in + B
  float A = 1.0f;
  cpx<float> B = {0.0f, 0.0f};
#pragma unroll
  for (int u = 0; u < S; ++u) {
    if (j0 + u >= ny) break;
    const float al = -a * m[u];
    B = {fmaf(al, B.x, d[u].x * m[u]), fmaf(al, B.y, d[u].y * m[u])};
    A *= al;
  }
  __syncthreads();
  sA[t][c] = A;
  sB[t][c] = B;
  __syncthreads();
  cpx<float> prev = {0.0f, 0.0f};
  for (int s = 0; s < t; ++s) {
    const float As = sA[s][c];
    const cpx<float> Bs = sB[s][c];
    prev = {fmaf(As, prev.x, Bs.x), fmaf(As, prev.y, Bs.y)};
  }
  // (the singular column holds its solution already: its maps are formed and
  // left unused, its replays skipped)
#pragma unroll
  for (int u = 0; u < S; ++u) {
    if (j0 + u >= ny || singular) break;
    cpx<float> v = d[u];
    v.x = (v.x - a * prev.x) * m[u];
    v.y = (v.y - a * prev.y) * m[u];
    d[u] = v;
    prev = v;
  }
  // back substitution x_j = xt_j - a m_j x_{j+1} (x_{ny-1} = xt_{ny-1}): this
  // segment's map from x at its upper end (j0 + S) to x_{j0}
  A = 1.0f;
  B = {0.0f, 0.0f};
#pragma unroll
  for (int u = S - 1; u >= 0; --u) {
    const int jj = j0 + u;
    if (jj >= ny) continue;
    if (jj == ny - 1) {
      A = 0.0f;
      B = d[u];
      continue;
    }
    const float cj = -a * m[u];
    B = {fmaf(cj, B.x, d[u].x), fmaf(cj, B.y, d[u].y)};
    A *= cj;
  }
  __syncthreads();
  sA[t][c] = A;
  sB[t][c] = B;
  __syncthreads();
  cpx<float> next = {0.0f, 0.0f};  // x at the segment's upper end
  for (int s = T - 1; s > t; --s) {
    const float As = sA[s][c];
    const cpx<float> Bs = sB[s][c];
    next = {fmaf(As, next.x, Bs.x), fmaf(As, next.y, Bs.y)};
  }
#pragma unroll
  for (int u = S - 1; u >= 0; --u) {
    const int jj = j0 + u;
    if (jj >= ny || singular) continue;
    cpx<float> v = d[u];
    if (jj < ny - 1) {
      const float cj = a * m[u];
      v.x -= cj * next.x;
      v.y -= cj * next.y;
    }
    d[u] = v;
    next = v;
  }
  if (valid) {
#pragma unroll
    for (int u = 0; u < S; ++u)
      if (j0 + u < ny) col[(size_t)(j0 + u) * nxh] = singular ? sline[j0 + u] : d[u];
  }
}

}  // namespace

// S: elements per thread, 16 S >= ny (S a power of two, at most 32)
int yscan_elems(int ny) {
  int s = 1;
  while (16 * s < ny) s *= 2;
  return s <= 32 ? s : 0;
}

cudaError_t launch_ythomas_scan(const GridDev& g, cpx<float>* spec, const float* tab, const int* line_off,
                                const int* line_len, float a, const DevScalars* zsc, cudaStream_t st) {
  const int nxh = g.nx / 2 + 1;
  const int grid = g.nz * ((nxh + 15) / 16);
  switch (yscan_elems(g.ny)) {
    case 1: k_ythomas_scan<1><<<grid, 256, 0, st>>>(g, spec, tab, line_off, line_len, a, zsc); break;
    case 2: k_ythomas_scan<2><<<grid, 256, 0, st>>>(g, spec, tab, line_off, line_len, a, zsc); break;
    case 4: k_ythomas_scan<4><<<grid, 256, 0, st>>>(g, spec, tab, line_off, line_len, a, zsc); break;
    case 8: k_ythomas_scan<8><<<grid, 256, 0, st>>>(g, spec, tab, line_off, line_len, a, zsc); break;
    case 16: k_ythomas_scan<16><<<grid, 256, 0, st>>>(g, spec, tab, line_off, line_len, a, zsc); break;
    case 32: k_ythomas_scan<32><<<grid, 256, 0, st>>>(g, spec, tab, line_off, line_len, a, zsc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ppe
