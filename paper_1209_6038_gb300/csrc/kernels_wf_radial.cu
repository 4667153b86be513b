// Wavefront FP64 kernels for the radial medium (one translation unit per variant).
#include "wavefront.cuh"

namespace ck {
CK_INSTANTIATE_WAVEFRONT(0)
}  // namespace ck
