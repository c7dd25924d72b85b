// Division by a run-time constant without the integer divide sequence:
// q = floor(x / d) = (x * m) >> p for 0 <= x < 2^31, with l = ceil(log2 d),
// p = 31 + l and m = ceil(2^p / d) < 2^32 (Granlund and Montgomery 1994,
// "Division by invariant integers using multiplication").  Built on the host.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define PPE_FD_HD __host__ __device__ __forceinline__
#else
#define PPE_FD_HD inline
#endif

namespace ppe {

struct FastDiv {
  uint32_t d;  // divisor (>= 1)
  uint32_t m;  // magic multiplier
  uint32_t p;  // total shift (31 .. 62)
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.p = 31 + l;
  const unsigned long long two_p = 1ull << f.p;
  f.m = (uint32_t)((two_p + d - 1) / d);
  return f;
}

PPE_FD_HD uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (uint32_t)(((unsigned long long)x * f.m) >> f.p);
}
PPE_FD_HD uint32_t fmod_(uint32_t x, const FastDiv& f) { return x - fdiv(x, f) * f.d; }

}  // namespace ppe
