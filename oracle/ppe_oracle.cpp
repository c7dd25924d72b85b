// FP64 reference implementation of the split pressure-gradient projection of
// Poblador-Ibanez & Sirignano (arXiv 2103.01874), Sec. 5.4, Eqs. (32)-(34), in
// plain single-threaded C++17.
//
// TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline leg load this library.  It shares no code with the CUDA path
// (nor with the numpy oracle beside it, against which it is cross-checked).
//
// What it computes (a direct solve, so the plain definition of the discrete
// result, step by step in the paper's order):
//   p_hat  = 2 p^n - p^{n-1}                                        Eq. (32)
//   rho_0  = min(rho)                                   text after Eq. (32)
//   f      = D[(1 - rho_0/rho_f) G p_hat] + (rho_0/dt)(D u* - S)   Eq. (34)
//   L p    = f - mean(f),  mean(p) = 0  (walls)                    Eq. (34)
//   u^{n+1} = u* - dt [G p / rho_0 + (1/rho_f - 1/rho_0) G p_hat]   Eq. (33)
// on the uniform staggered mesh (Sec. 5; "standard finite-volume
// techniques", paragraph after Eq. (34)): G cell -> face differences (zero on
// the wall faces of y), D face -> cell divergence, L = D G the 7-point
// operator; rho_f the arithmetic (or harmonic) mean of the two cells.
//
// The solve (the fast Poisson solver stated after Eq. (34)) with transforms of
// its own:
//   * complex DFT of any length by recursive Cooley-Tukey decimation in time
//     (radix 2 and 3, a direct sum for any other factor), unscaled forward,
//     the inverse with exp(+2 pi i/N);
//   * the real DFT along x as the complex DFT of the real line (kx = 0..nx/2),
//     its inverse through the Hermitian completion of the spectrum;
//   * in y, per wavenumber pair (kx, kz), the tridiagonal system of the
//     7-point operator with the x and z second differences replaced by their
//     eigenvalues lam_x + lam_z, lam_x = -(4/dx^2) sin^2(pi kx/nx), solved by
//     the Thomas algorithm; the singular line kx = kz = 0 (walls) by pinning
//     its first value and removing the mean afterwards (zero-mean solution).
//     A second y method -- DCT-II, divide by lam_x + lam_y + lam_z with
//     lam_y = -(4/dy^2) sin^2(pi ky/(2 ny)), DCT-III -- exists for
//     cross-checks (walls only).
// Outflow top (p = 0 on the face y = Ly, ghost p_ny = -p_{ny-1}): the last
// diagonal of the y system is -3a + lam, every line is regular, and the top
// face's G is (0 - q_{ny-1}) / (dy/2).
#include <math.h>
#include <stddef.h>

#include <algorithm>
#include <complex>
#include <type_traits>
#include <vector>

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;

struct Grid {
  int nx, ny, nz;
  double dx, dy, dz;
  size_t cell(int i, int j, int k) const { return ((size_t)k * ny + j) * nx + i; }
  size_t vface(int i, int j, int k) const { return ((size_t)k * (ny + 1) + j) * nx + i; }
  size_t n() const { return (size_t)nx * ny * nz; }
  size_t nv() const { return (size_t)nx * (ny + 1) * nz; }
};

// ---------------------------------------------------------------------------
// transforms
// ---------------------------------------------------------------------------
// exp(sign 2 pi i t / n), t reduced modulo n first
cd root(long t, long n, int sign) {
  t %= n;
  if (t < 0) t += n;
  const double a = 2.0 * kPi * (double)t / (double)n;
  return cd(cos(a), sign * sin(a));
}

// X_k = sum_m x_{m s} exp(sign 2 pi i k m / n), the n values x[0], x[s], ...
void dft_direct_strided(int n, int sign, const cd* x, int s, cd* X) {
  for (int k = 0; k < n; ++k) {
    cd acc = 0.0;
    for (int m = 0; m < n; ++m) acc += x[(size_t)m * s] * root((long)k * m, n, sign);
    X[k] = acc;
  }
}

// Decimation in time: for a factor r of n (2 or 3), the r subsequences
// x[q + r t] (t < n/r) are transformed, then combined:
//   X[k + m s] = sum_q exp(sign 2 pi i q (k + m s) / n) Sub_q[k],  m = n / r.
void fft_strided(int n, int sign, const cd* x, int s, cd* X) {
  if (n == 1) {
    X[0] = x[0];
    return;
  }
  const int r = (n % 2 == 0) ? 2 : ((n % 3 == 0) ? 3 : 0);
  if (r == 0) {
    dft_direct_strided(n, sign, x, s, X);
    return;
  }
  const int m = n / r;
  std::vector<cd> sub((size_t)n);
  for (int q = 0; q < r; ++q) fft_strided(m, sign, x + (size_t)q * s, s * r, &sub[(size_t)q * m]);
  for (int k = 0; k < m; ++k)
    for (int b = 0; b < r; ++b) {
      cd acc = 0.0;
      for (int q = 0; q < r; ++q) acc += sub[(size_t)q * m + k] * root((long)q * (k + (long)m * b), n, sign);
      X[k + (size_t)m * b] = acc;
    }
}

void fft(std::vector<cd>& a, int sign) {
  std::vector<cd> out(a.size());
  fft_strided((int)a.size(), sign, a.data(), 1, out.data());
  a.swap(out);
}

// DCT-II  X_k = sum_j x_j cos(pi k (j + 1/2) / n), from the 2n-point DFT of the
// even extension y = (x_0 .. x_{n-1}, x_{n-1} .. x_0):
//   Y_k = exp(i pi k / (2n)) 2 X_k.
template <typename V>
void dct2_fft(int n, const V* x, V* X) {
  auto part = [](const V& v, int which) -> double {
    if constexpr (std::is_same<V, cd>::value) return which ? v.imag() : v.real();
    else return which ? 0.0 : (double)v;
  };
  std::vector<cd> yr(2 * (size_t)n), yi(2 * (size_t)n);
  for (int j = 0; j < n; ++j) {
    yr[j] = yr[2 * (size_t)n - 1 - j] = part(x[j], 0);
    yi[j] = yi[2 * (size_t)n - 1 - j] = part(x[j], 1);
  }
  fft(yr, -1);
  fft(yi, -1);
  for (int k = 0; k < n; ++k) {
    const cd w = root(-(long)k, 4 * (long)n, 1) * 0.5;  // exp(-i pi k/(2n)) / 2
    const double a = (w * yr[k]).real(), b = (w * yi[k]).real();
    if constexpr (std::is_same<V, cd>::value) X[k] = cd(a, b);
    else X[k] = a;
  }
}

// DCT-III, the inverse of dct2:  x_j = (1/n) X_0 + (2/n) sum_{k>=1} X_k cos(pi k (j + 1/2)/n)
template <typename V>
void dct3_direct(int n, const V* X, V* x) {
  for (int j = 0; j < n; ++j) {
    V acc = X[0] * (1.0 / n);
    for (int k = 1; k < n; ++k) acc += X[k] * ((2.0 / n) * cos(kPi * k * (j + 0.5) / n));
    x[j] = acc;
  }
}

// Thomas algorithm: sub[j] x_{j-1} + diag[j] x_j + sup[j] x_{j+1} = d_j
// (sub[0], sup[n-1] unused); forward elimination, back substitution.
template <typename V>
void thomas(int n, const double* sub, const double* diag, const double* sup, const V* d, V* x) {
  std::vector<double> cp((size_t)n);
  std::vector<V> dp((size_t)n);
  double piv = diag[0];
  cp[0] = n > 1 ? sup[0] / piv : 0.0;
  dp[0] = d[0] / piv;
  for (int j = 1; j < n; ++j) {
    piv = diag[j] - sub[j] * cp[j - 1];
    cp[j] = j + 1 < n ? sup[j] / piv : 0.0;
    dp[j] = (d[j] - sub[j] * dp[j - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int j = n - 2; j >= 0; --j) x[j] = dp[j] - cp[j] * x[j + 1];
}

// ---------------------------------------------------------------------------
// staggered-mesh operators
// ---------------------------------------------------------------------------
// G q: x faces gx[i] = (q_i - q_{i-1})/dx (periodic), z alike, y faces
// gy[j] = (q_j - q_{j-1})/dy for 0 < j < ny; 0 on the walls; an outflow top
// face sees q = 0 half a cell above the last centre.
void grad(const Grid& g, const std::vector<double>& q, int top_open, std::vector<double>& gx, std::vector<double>& gy,
          std::vector<double>& gz) {
  gx.assign(g.n(), 0.0);
  gz.assign(g.n(), 0.0);
  gy.assign(g.nv(), 0.0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t c = g.cell(i, j, k);
        gx[c] = (q[c] - q[g.cell((i + g.nx - 1) % g.nx, j, k)]) / g.dx;
        gz[c] = (q[c] - q[g.cell(i, j, (k + g.nz - 1) % g.nz)]) / g.dz;
        if (j > 0) gy[g.vface(i, j, k)] = (q[c] - q[g.cell(i, j - 1, k)]) / g.dy;
      }
  if (top_open)
    for (int k = 0; k < g.nz; ++k)
      for (int i = 0; i < g.nx; ++i) gy[g.vface(i, g.ny, k)] = (0.0 - q[g.cell(i, g.ny - 1, k)]) / (0.5 * g.dy);
}

// D (a, b, c) at cell (i, j, k) = (a_{i+1} - a_i)/dx + (b_{j+1} - b_j)/dy + (c_{k+1} - c_k)/dz
void divergence(const Grid& g, const std::vector<double>& a, const std::vector<double>& b, const std::vector<double>& c,
                std::vector<double>& out) {
  out.assign(g.n(), 0.0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t cc = g.cell(i, j, k);
        out[cc] = (a[g.cell((i + 1) % g.nx, j, k)] - a[cc]) / g.dx +
                  (b[g.vface(i, j + 1, k)] - b[g.vface(i, j, k)]) / g.dy +
                  (c[g.cell(i, j, (k + 1) % g.nz)] - c[cc]) / g.dz;
      }
}

// face density of the face between cells with densities r0, r1
double face_rho(double r0, double r1, int rule) { return rule == 0 ? 0.5 * (r0 + r1) : 2.0 / (1.0 / r0 + 1.0 / r1); }

// face densities on the x, y and z faces (a wall face gets its one cell's
// value; G vanishes there, so it is never used; the outflow top face gets the
// top cell's, as if the ghost cell had the same density)
void face_densities(const Grid& g, const double* rho, int rule, std::vector<double>& rx, std::vector<double>& ry,
                    std::vector<double>& rz) {
  rx.assign(g.n(), 0.0);
  rz.assign(g.n(), 0.0);
  ry.assign(g.nv(), 0.0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        if (j < g.ny) {
          const size_t c = g.cell(i, j, k);
          rx[c] = face_rho(rho[g.cell((i + g.nx - 1) % g.nx, j, k)], rho[c], rule);
          rz[c] = face_rho(rho[g.cell(i, j, (k + g.nz - 1) % g.nz)], rho[c], rule);
        }
        const double lo = rho[g.cell(i, j > 0 ? j - 1 : 0, k)], hi = rho[g.cell(i, j < g.ny ? j : g.ny - 1, k)];
        ry[g.vface(i, j, k)] = (j == 0) ? hi : (j == g.ny ? lo : face_rho(lo, hi, rule));
      }
}

// Planted mistakes for the tests of the pins (0: none): 1 the y diagonal's
// sign flipped, 2 the split term of Eq. (34) dropped, 3 S added instead of
// subtracted.
struct Mutation {
  int m;
};

// Eq. (34)
void rhs(const Grid& g, const double* u, const double* v, const double* w, const double* S, const double* rho,
         const double* pn, const double* pnm1, double rho0, double dt, int rule, int top_open, Mutation mut,
         std::vector<double>& f) {
  std::vector<double> ph(g.n());
  for (size_t c = 0; c < g.n(); ++c) ph[c] = 2.0 * pn[c] - pnm1[c];  // Eq. (32)
  std::vector<double> gx, gy, gz, rx, ry, rz;
  grad(g, ph, top_open, gx, gy, gz);
  face_densities(g, rho, rule, rx, ry, rz);
  for (size_t c = 0; c < g.n(); ++c) {
    gx[c] *= 1.0 - rho0 / rx[c];
    gz[c] *= 1.0 - rho0 / rz[c];
  }
  for (size_t c = 0; c < g.nv(); ++c) gy[c] *= 1.0 - rho0 / ry[c];
  std::vector<double> split, du;
  divergence(g, gx, gy, gz, split);
  std::vector<double> uu(u, u + g.n()), vv(v, v + g.nv()), ww(w, w + g.n());
  divergence(g, uu, vv, ww, du);
  f.assign(g.n(), 0.0);
  for (size_t c = 0; c < g.n(); ++c) {
    const double s = mut.m == 3 ? -S[c] : S[c];
    f[c] = (mut.m == 2 ? 0.0 : split[c]) + (rho0 / dt) * (du[c] - s);
  }
}

// Solve L p = f (- mean f for walls) with mean(p) = 0 (walls), by DFT in x and
// z and a tridiagonal (Thomas) or cosine-transform solve in y.
void solve(const Grid& g, const double* f, int top_open, int y_method, Mutation mut, std::vector<double>& p) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxh = nx / 2 + 1;
  double fm = 0.0;
  if (!top_open) {
    for (size_t c = 0; c < g.n(); ++c) fm += f[c];
    fm /= (double)g.n();
  }
  // spectrum [k][j][kx], then [kz][j][kx] after the z transforms
  std::vector<cd> spec((size_t)nz * ny * nxh);
  std::vector<cd> line;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      line.assign(nx, 0.0);
      for (int i = 0; i < nx; ++i) line[i] = f[g.cell(i, j, k)] - fm;
      fft(line, -1);
      for (int kx = 0; kx < nxh; ++kx) spec[((size_t)k * ny + j) * nxh + kx] = line[kx];
    }
  for (int j = 0; j < ny; ++j)
    for (int kx = 0; kx < nxh; ++kx) {
      line.assign(nz, 0.0);
      for (int k = 0; k < nz; ++k) line[k] = spec[((size_t)k * ny + j) * nxh + kx];
      fft(line, -1);
      for (int k = 0; k < nz; ++k) spec[((size_t)k * ny + j) * nxh + kx] = line[k];
    }
  // y: per (kx, kz)
  const double a = 1.0 / (g.dy * g.dy);
  std::vector<double> sub(ny, a), sup(ny, a), diag(ny);
  std::vector<cd> d(ny), x(ny);
  for (int kz = 0; kz < nz; ++kz)
    for (int kx = 0; kx < nxh; ++kx) {
      const double sx = sin(kPi * kx / nx), sz = sin(kPi * kz / nz);
      const double lam = -(4.0 / (g.dx * g.dx)) * sx * sx - (4.0 / (g.dz * g.dz)) * sz * sz;
      for (int j = 0; j < ny; ++j) d[j] = spec[((size_t)kz * ny + j) * nxh + kx];
      const bool singular = !top_open && kx == 0 && kz == 0;
      if (y_method == 1 && !top_open) {
        // DCT-II, divide by the eigenvalues (zero mode dropped), DCT-III
        std::vector<cd> X(ny);
        dct2_fft(ny, d.data(), X.data());
        for (int ky = 0; ky < ny; ++ky) {
          const double sy = sin(kPi * ky / (2.0 * ny));
          const double l = lam - (4.0 / (g.dy * g.dy)) * sy * sy;
          X[ky] = (singular && ky == 0) ? cd(0.0) : X[ky] / l;
        }
        dct3_direct(ny, X.data(), x.data());
      } else {
        const double sgn = mut.m == 1 ? -1.0 : 1.0;  // planted mistake 1
        for (int j = 0; j < ny; ++j) diag[j] = sgn * -2.0 * a + lam;
        diag[0] = sgn * -a + lam;
        diag[ny - 1] = (top_open ? -3.0 * sgn * a : -sgn * a) + lam;
        if (!singular) {
          thomas(ny, sub.data(), diag.data(), sup.data(), d.data(), x.data());
        } else {
          // the constant line: pin x_0 = 0, solve rows 1 .. ny-1, remove the mean
          x[0] = 0.0;
          if (ny > 1) thomas(ny - 1, sub.data() + 1, diag.data() + 1, sup.data() + 1, d.data() + 1, x.data() + 1);
          cd mean = 0.0;
          for (int j = 0; j < ny; ++j) mean += x[j];
          mean /= (double)ny;
          for (int j = 0; j < ny; ++j) x[j] -= mean;
        }
      }
      for (int j = 0; j < ny; ++j) spec[((size_t)kz * ny + j) * nxh + kx] = x[j];
    }
  // inverse z, inverse x (Hermitian completion), 1/(nx nz)
  for (int j = 0; j < ny; ++j)
    for (int kx = 0; kx < nxh; ++kx) {
      line.assign(nz, 0.0);
      for (int k = 0; k < nz; ++k) line[k] = spec[((size_t)k * ny + j) * nxh + kx];
      fft(line, 1);
      for (int k = 0; k < nz; ++k) spec[((size_t)k * ny + j) * nxh + kx] = line[k];
    }
  p.assign(g.n(), 0.0);
  const double scale = 1.0 / ((double)nx * (double)nz);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      line.assign(nx, 0.0);
      for (int kx = 0; kx < nxh; ++kx) line[kx] = spec[((size_t)k * ny + j) * nxh + kx];
      for (int kx = nxh; kx < nx; ++kx) line[kx] = std::conj(line[nx - kx]);
      fft(line, 1);
      for (int i = 0; i < nx; ++i) p[g.cell(i, j, k)] = scale * line[i].real();
    }
}

// Eq. (33): u^{n+1} = u* - dt [G p / rho_0 + (1/rho_f - 1/rho_0) G p_hat];
// the wall faces of v keep v* (G = 0 there)
void correct(const Grid& g, const double* u, const double* v, const double* w, const double* rho, const double* p,
             const double* pn, const double* pnm1, double rho0, double dt, int rule, int top_open, double* u1,
             double* v1, double* w1) {
  std::vector<double> pp(p, p + g.n()), ph(g.n());
  for (size_t c = 0; c < g.n(); ++c) ph[c] = 2.0 * pn[c] - pnm1[c];
  std::vector<double> gpx, gpy, gpz, ghx, ghy, ghz, rx, ry, rz;
  grad(g, pp, top_open, gpx, gpy, gpz);
  grad(g, ph, top_open, ghx, ghy, ghz);
  face_densities(g, rho, rule, rx, ry, rz);
  for (size_t c = 0; c < g.n(); ++c) {
    u1[c] = u[c] - dt * (gpx[c] / rho0 + (1.0 / rx[c] - 1.0 / rho0) * ghx[c]);
    w1[c] = w[c] - dt * (gpz[c] / rho0 + (1.0 / rz[c] - 1.0 / rho0) * ghz[c]);
  }
  for (size_t c = 0; c < g.nv(); ++c) v1[c] = v[c] - dt * (gpy[c] / rho0 + (1.0 / ry[c] - 1.0 / rho0) * ghy[c]);
}

bool grid_ok(int nx, int ny, int nz, double lx, double ly, double lz) {
  return nx >= 2 && ny >= 2 && nz >= 1 && nx % 2 == 0 && lx > 0 && ly > 0 && lz > 0;
}

Grid make_grid(int nx, int ny, int nz, double lx, double ly, double lz) {
  return Grid{nx, ny, nz, lx / nx, ly / ny, lz / nz};
}

}  // namespace

extern "C" {

int oracle_version(void) { return 1; }

// The whole projection: f, p (mean zero for walls), u^{n+1}, v^{n+1}, w^{n+1}
// and the rho_0 used (min(rho) when rho0 <= 0).  face_rule 0 arithmetic, 1
// harmonic; bc_top 0 wall, 1 outflow; y_method 0 Thomas, 1 cosine transform
// (walls); mutation 0 (others plant a mistake, for the pins' tests).
// Returns 0, or -1 on invalid arguments.
int oracle_project(int nx, int ny, int nz, double lx, double ly, double lz, int face_rule, int bc_top, int y_method,
                   const double* u, const double* v, const double* w, const double* S, const double* rho,
                   const double* p_n, const double* p_nm1, double rho0, double dt, int mutation, double* f, double* p,
                   double* u_out, double* v_out, double* w_out, double* rho0_used) {
  if (!grid_ok(nx, ny, nz, lx, ly, lz) || !(dt > 0) || !u || !v || !w || !S || !rho || !p_n || !p_nm1 || !f || !p ||
      !u_out || !v_out || !w_out)
    return -1;
  const Grid g = make_grid(nx, ny, nz, lx, ly, lz);
  if (!(rho0 > 0)) rho0 = *std::min_element(rho, rho + g.n());
  if (rho0_used) *rho0_used = rho0;
  std::vector<double> fv, pv;
  rhs(g, u, v, w, S, rho, p_n, p_nm1, rho0, dt, face_rule, bc_top, Mutation{mutation}, fv);
  solve(g, fv.data(), bc_top, y_method, Mutation{mutation}, pv);
  correct(g, u, v, w, rho, pv.data(), p_n, p_nm1, rho0, dt, face_rule, bc_top, u_out, v_out, w_out);
  std::copy(fv.begin(), fv.end(), f);
  std::copy(pv.begin(), pv.end(), p);
  return 0;
}

// Eq. (34) alone
int oracle_rhs(int nx, int ny, int nz, double lx, double ly, double lz, int face_rule, int bc_top, const double* u,
               const double* v, const double* w, const double* S, const double* rho, const double* p_n,
               const double* p_nm1, double rho0, double dt, double* f) {
  if (!grid_ok(nx, ny, nz, lx, ly, lz) || !(dt > 0) || !(rho0 > 0) || !f) return -1;
  const Grid g = make_grid(nx, ny, nz, lx, ly, lz);
  std::vector<double> fv;
  rhs(g, u, v, w, S, rho, p_n, p_nm1, rho0, dt, face_rule, bc_top, Mutation{0}, fv);
  std::copy(fv.begin(), fv.end(), f);
  return 0;
}

// L p = f (- mean f for walls), mean(p) = 0 for walls
int oracle_solve(int nx, int ny, int nz, double lx, double ly, double lz, int bc_top, int y_method, const double* f,
                 double* p) {
  if (!grid_ok(nx, ny, nz, lx, ly, lz) || !f || !p) return -1;
  const Grid g = make_grid(nx, ny, nz, lx, ly, lz);
  std::vector<double> pv;
  solve(g, f, bc_top, y_method, Mutation{0}, pv);
  std::copy(pv.begin(), pv.end(), p);
  return 0;
}

// L q = D G q (the 7-point operator)
int oracle_laplacian(int nx, int ny, int nz, double lx, double ly, double lz, int bc_top, const double* q,
                     double* out) {
  if (!grid_ok(nx, ny, nz, lx, ly, lz) || !q || !out) return -1;
  const Grid g = make_grid(nx, ny, nz, lx, ly, lz);
  std::vector<double> qq(q, q + g.n()), gx, gy, gz, d;
  grad(g, qq, bc_top, gx, gy, gz);
  divergence(g, gx, gy, gz, d);
  std::copy(d.begin(), d.end(), out);
  return 0;
}

// building blocks, for the brute-force pins
int oracle_fft(int n, int sign, const double* re, const double* im, double* ore, double* oim) {
  if (n < 1 || (sign != 1 && sign != -1)) return -1;
  std::vector<cd> a((size_t)n);
  for (int k = 0; k < n; ++k) a[k] = cd(re[k], im[k]);
  fft(a, sign);
  for (int k = 0; k < n; ++k) {
    ore[k] = a[k].real();
    oim[k] = a[k].imag();
  }
  return 0;
}

int oracle_dft_direct(int n, int sign, const double* re, const double* im, double* ore, double* oim) {
  if (n < 1 || (sign != 1 && sign != -1)) return -1;
  std::vector<cd> a((size_t)n), b((size_t)n);
  for (int k = 0; k < n; ++k) a[k] = cd(re[k], im[k]);
  dft_direct_strided(n, sign, a.data(), 1, b.data());
  for (int k = 0; k < n; ++k) {
    ore[k] = b[k].real();
    oim[k] = b[k].imag();
  }
  return 0;
}

int oracle_dct2(int n, const double* x, double* X) {
  if (n < 1) return -1;
  dct2_fft(n, x, X);
  return 0;
}

int oracle_dct3(int n, const double* X, double* x) {
  if (n < 1) return -1;
  dct3_direct(n, X, x);
  return 0;
}

int oracle_thomas(int n, const double* sub, const double* diag, const double* sup, const double* d, double* x) {
  if (n < 1) return -1;
  thomas(n, sub, diag, sup, d, x);
  return 0;
}

}  // extern "C"
