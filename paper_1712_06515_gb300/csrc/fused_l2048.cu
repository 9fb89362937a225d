// Fused kernel instantiations for coset lengths 2048.
#include "fused_kernel.cuh"

namespace cc {
CC_FUSED_INSTANTIATE(2048)
}  // namespace cc
