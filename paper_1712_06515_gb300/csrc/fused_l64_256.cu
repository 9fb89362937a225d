// Fused kernel instantiations for coset lengths 64, 128, 256.
#include "fused_kernel.cuh"

namespace cc {
CC_FUSED_INSTANTIATE(64)
CC_FUSED_INSTANTIATE(128)
CC_FUSED_INSTANTIATE(256)
}  // namespace cc
