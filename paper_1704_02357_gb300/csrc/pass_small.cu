// Transform passes instantiated for mesh sides: 16 32 64 128.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(16)
PSPEC_DEFINE_PASSES(32)
PSPEC_DEFINE_PASSES(64)
PSPEC_DEFINE_PASSES(128)
}  // namespace pspec
