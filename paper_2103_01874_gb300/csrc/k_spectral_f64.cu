// Spectral passes of the direct Poisson solve (paragraph after Eq. (34)) in
// FP64 (the FP64 form with an outflow top: its tridiagonal y solve).
#include "spectral.cuh"

namespace ppe {
PPE_INST(double)
}  // namespace ppe
