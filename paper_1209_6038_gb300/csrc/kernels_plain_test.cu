// Plain FP64 kernels for the test medium (one translation unit per variant).
#include "kernels_plain.cuh"

namespace ck {
CK_INSTANTIATE_PLAIN(2)
}  // namespace ck
