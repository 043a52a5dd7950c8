// Transform passes instantiated for mesh sides: 1024.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(1024)
}  // namespace pspec
