// Spectral passes of the direct Poisson solve (paragraph after Eq. (34)) in
// FP32 (the refinement form's solves).
#include "spectral.cuh"

namespace ppe {
PPE_INST(float)
}  // namespace ppe
