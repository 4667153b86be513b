// Plain FP64 kernels for the radial medium (one translation unit per variant).
#include "kernels_plain.cuh"

namespace ck {
CK_INSTANTIATE_PLAIN(0)
}  // namespace ck
