// Transform passes instantiated for mesh sides: 256.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(256)
}  // namespace pspec
