// Fused kernel instantiations for coset lengths 512, 1024.
#include "fused_kernel.cuh"

namespace cc {
CC_FUSED_INSTANTIATE(512)
CC_FUSED_INSTANTIATE(1024)
}  // namespace cc
