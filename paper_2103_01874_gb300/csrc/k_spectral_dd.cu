// Spectral passes of the direct Poisson solve (paragraph after Eq. (34)) in
// double-float pairs (the FP64 form with walls: transforms and the cosine-transform y solve on the FP32 pipe).
#include "spectral.cuh"

namespace ppe {
PPE_INST(dd)
}  // namespace ppe
