// Plain FP64 kernels for the azimuthal medium (one translation unit per variant).
#include "kernels_plain.cuh"

namespace ck {
CK_INSTANTIATE_PLAIN(1)
}  // namespace ck
