// Fused kernel instantiations for coset lengths 4096.
#include "fused_kernel.cuh"

namespace cc {
CC_FUSED_INSTANTIATE(4096)
}  // namespace cc
