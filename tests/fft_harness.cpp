// Host emulation of the shared-memory Stockham FFT (paper_2103_01874_gb300/
// csrc/fft.cuh): the threads of one CTA run one after another, which is exact
// for these passes (each reads one buffer and writes the other, with a barrier
// between passes).  Prints the max error against a naive long-double DFT,
// relative to the largest output.  Driven by test_host_kernels.py.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <utility>
#include <vector>

struct Dim3 { unsigned x, y, z; };
static Dim3 threadIdx = {0, 0, 0};
static Dim3 blockDim = {256, 1, 1};
static inline void __syncthreads() {}

#include "fft.cuh"

using namespace ppe;

static RadixPlan plan_for(int n, int maxr) {
  RadixPlan rp{};
  rp.n = n;
  int m = n;
  while (maxr >= 16 && m % 16 == 0) { rp.r[rp.nst++] = 16; m /= 16; }
  if (maxr >= 8 && m % 8 == 0) { rp.r[rp.nst++] = 8; m /= 8; }
  if (m % 4 == 0) { rp.r[rp.nst++] = 4; m /= 4; }
  while (m % 4 == 0) { rp.r[rp.nst++] = 4; m /= 4; }
  if (m % 2 == 0) { rp.r[rp.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { rp.r[rp.nst++] = 3; m /= 3; }
  int ns = 1;
  for (int s = 0; s < rp.nst; ++s) { rp.ns[s] = make_fastdiv(ns); ns *= rp.r[s]; }
  return rp;
}

template <typename T, bool INV, int N, int MAXR>
static void ct_passes(cpx<T>*& A, cpx<T>*& B, int nl_log2, int ls, int es, const cpx<T>* tw) {
  // the passes of fft_lines_ct with the CTA's threads run in turn
  constexpr int S = ctfft::nst(N, MAXR);
  auto one = [&](auto sc) {
    constexpr int s = decltype(sc)::value;
    for (unsigned t = 0; t < blockDim.x; ++t) {
      threadIdx.x = t;
      ctfft::pass_ct<T, INV, N, s, MAXR, 1>(A, B, nl_log2, ls, es, tw);
    }
    std::swap(A, B);
  };
  [&]<int... I>(std::integer_sequence<int, I...>) { (one(std::integral_constant<int, I>{}), ...); }
  (std::make_integer_sequence<int, S>{});
}

template <typename T, bool INV>
static bool run_ct(int n, int maxr, cpx<T>*& A, cpx<T>*& B, int nl_log2, int ls, int es, const cpx<T>* tw) {
#define PPE_CT(NN)                                                             \
  if (n == NN) {                                                               \
    if (maxr == 16) ct_passes<T, INV, NN, 16>(A, B, nl_log2, ls, es, tw);      \
    else ct_passes<T, INV, NN, 8>(A, B, nl_log2, ls, es, tw);                  \
    return true;                                                               \
  }
  PPE_CT(16) PPE_CT(24) PPE_CT(32) PPE_CT(48) PPE_CT(64) PPE_CT(96) PPE_CT(128) PPE_CT(192) PPE_CT(256) PPE_CT(384)
#undef PPE_CT
  return false;
}

static bool g_ct = false;

template <typename T, bool INV>
static double run(int n, int nl, int ls, int es, int maxr, unsigned seed) {
  srand(seed);
  const int size = (nl - 1) * ls + (n - 1) * es + 1;
  std::vector<cpx<T>> a(size), b(size), tw(n);
  std::vector<std::complex<long double>> x((size_t)nl * n);
  for (int l = 0; l < nl; ++l)
    for (int e = 0; e < n; ++e) {
      const double re = rand() / (double)RAND_MAX - 0.5, im = rand() / (double)RAND_MAX - 0.5;
      a[l * ls + e * es] = {(T)re, (T)im};
      x[(size_t)l * n + e] = {(long double)(T)re, (long double)(T)im};
    }
  const long double PI = 3.141592653589793238462643383279503L;
  for (int t = 0; t < n; ++t) tw[t] = {(T)cosl(2 * PI * t / n), (T)(-sinl(2 * PI * t / n))};
  RadixPlan rp = plan_for(n, maxr);
  int nl_log2 = 0;
  while ((1 << nl_log2) < nl) ++nl_log2;
  cpx<T>* A = a.data();
  cpx<T>* B = b.data();
  // fft_lines with the threads of the CTA run in turn inside each pass
  int Ns = 1;
  if (g_ct && !run_ct<T, INV>(n, maxr, A, B, nl_log2, ls, es, tw.data())) return -1.0;
  for (int s = 0; s < (g_ct ? 0 : rp.nst); ++s) {
    for (unsigned t = 0; t < blockDim.x; ++t) {
      threadIdx.x = t;
      switch (rp.r[s]) {
        case 16: stockham_pass<T, INV, 16>(A, B, nl_log2, n, ls, es, Ns, rp.ns[s], tw.data(), 1); break;
        case 8: stockham_pass<T, INV, 8>(A, B, nl_log2, n, ls, es, Ns, rp.ns[s], tw.data(), 1); break;
        case 4: stockham_pass<T, INV, 4>(A, B, nl_log2, n, ls, es, Ns, rp.ns[s], tw.data(), 1); break;
        case 2: stockham_pass<T, INV, 2>(A, B, nl_log2, n, ls, es, Ns, rp.ns[s], tw.data(), 1); break;
        default: stockham_pass<T, INV, 3>(A, B, nl_log2, n, ls, es, Ns, rp.ns[s], tw.data(), 1); break;
      }
    }
    std::swap(A, B);
    Ns *= rp.r[s];
  }
  long double err = 0, mx = 0;
  const long double sg = INV ? 1 : -1;
  for (int l = 0; l < nl; ++l)
    for (int k = 0; k < n; ++k) {
      std::complex<long double> want = 0;
      for (int e = 0; e < n; ++e) {
        const long double ang = sg * 2 * PI * (long double)((long long)e * k % n) / n;
        want += x[(size_t)l * n + e] * std::complex<long double>(cosl(ang), sinl(ang));
      }
      const cpx<T> g = A[l * ls + k * es];
      err = std::max(err, std::abs(std::complex<long double>(g.x, g.y) - want));
      mx = std::max(mx, std::abs(want));
    }
  return (double)(err / mx);
}

int main(int argc, char** argv) {
  // args: type(f|d) inv(0|1) n nl ls es maxr [ct]
  if (argc < 8) return 2;
  g_ct = argc > 8 && argv[8][0] == 'c';
  const bool dbl = argv[1][0] == 'd';
  const int inv = atoi(argv[2]), n = atoi(argv[3]), nl = atoi(argv[4]), ls = atoi(argv[5]), es = atoi(argv[6]),
            maxr = atoi(argv[7]);
  double e;
  if (dbl) e = inv ? run<double, true>(n, nl, ls, es, maxr, 7) : run<double, false>(n, nl, ls, es, maxr, 7);
  else e = inv ? run<float, true>(n, nl, ls, es, maxr, 7) : run<float, false>(n, nl, ls, es, maxr, 7);
  printf("%.3e\n", e);
  return 0;
}
