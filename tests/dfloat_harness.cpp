// Host harness for paper_2103_01874_gb300/csrc/dfloat.cuh and fastdiv.cuh:
// reads commands on stdin, prints results (floats as C99 hex).  Built and
// driven by test_dfloat.py.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "dfloat.cuh"
#include "fastdiv.cuh"

using namespace ppe;

int main() {
  char op[16];
  while (std::scanf("%15s", op) == 1) {
    if (!std::strcmp(op, "fastdiv")) {
      // fastdiv d x0 count stride: prints the number of mismatches
      unsigned d, x0, count, stride;
      std::scanf("%u %u %u %u", &d, &x0, &count, &stride);
      const FastDiv f = make_fastdiv(d);
      unsigned long bad = 0;
      for (unsigned long c = 0; c < count; ++c) {
        const unsigned long x = x0 + c * (unsigned long)stride;
        if (x >= (1ul << 31)) break;
        if (fdiv((uint32_t)x, f) != (uint32_t)(x / d) || fmod_((uint32_t)x, f) != (uint32_t)(x % d)) ++bad;
      }
      std::printf("%lu\n", bad);
    } else if (!std::strcmp(op, "d2df")) {
      double x;
      std::scanf("%la", &x);
      df r = d2df(x);
      std::printf("%a %a\n", (double)r.hi, (double)r.lo);
    } else if (!std::strcmp(op, "df2d") || !std::strcmp(op, "df2d_alu")) {
      double h, l;
      std::scanf("%la %la", &h, &l);
      const df a{(float)h, (float)l};
      std::printf("%a\n", op[4] ? df2d_alu(a) : df2d(a));
    } else if (!std::strcmp(op, "dot2sub") || !std::strcmp(op, "dot2add")) {
      // a b -+ c d for four pairs
      double v[8];
      for (int i = 0; i < 8; ++i) std::scanf("%la", &v[i]);
      const dd a((float)v[0], (float)v[1]), b((float)v[2], (float)v[3]), c((float)v[4], (float)v[5]),
          d((float)v[6], (float)v[7]);
      const dd r = op[4] == 's' ? dd_dot2<true>(a, b, c, d) : dd_dot2<false>(a, b, c, d);
      std::printf("%a %a\n", (double)r.hi, (double)r.lo);
    } else if (!std::strcmp(op, "addlazy")) {
      // a + b + c with lazy adds, then one normalisation
      double v[6];
      for (int i = 0; i < 6; ++i) std::scanf("%la", &v[i]);
      const dd a((float)v[0], (float)v[1]), b((float)v[2], (float)v[3]), c((float)v[4], (float)v[5]);
      const dd r = dd_norm(dd_add_lazy(dd_add_lazy(a, b), c));
      std::printf("%a %a\n", (double)r.hi, (double)r.lo);
    } else {
      double ah, al, bh, bl;
      std::scanf("%la %la %la %la", &ah, &al, &bh, &bl);
      df a{(float)ah, (float)al}, b{(float)bh, (float)bl}, r;
      if (!std::strcmp(op, "add")) r = df_add(a, b);
      else if (!std::strcmp(op, "sub")) r = df_sub(a, b);
      else if (!std::strcmp(op, "mul")) r = df_mul(a, b);
      else if (!std::strcmp(op, "mulf")) r = df_mul_f(a, b.hi);
      else if (!std::strcmp(op, "recip")) r = df_recip(a);
      else return 2;
      std::printf("%a %a\n", (double)r.hi, (double)r.lo);
    }
  }
  return 0;
}
