// Transform passes instantiated for mesh sides: 512.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(512)
}  // namespace pspec
