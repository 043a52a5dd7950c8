// Transform passes instantiated for mesh sides: 384.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(384)
}  // namespace pspec
