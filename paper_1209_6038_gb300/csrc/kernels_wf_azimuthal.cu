// Wavefront FP64 kernels for the azimuthal medium (one translation unit per variant).
#include "wavefront.cuh"

namespace ck {
CK_INSTANTIATE_WAVEFRONT(1)
}  // namespace ck
