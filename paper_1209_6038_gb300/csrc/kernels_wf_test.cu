// Wavefront FP64 kernels for the test medium (one translation unit per variant).
#include "wavefront.cuh"

namespace ck {
CK_INSTANTIATE_WAVEFRONT(2)
}  // namespace ck
