// Transform passes instantiated for mesh sides: 48 96 192.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(48)
PSPEC_DEFINE_PASSES(96)
PSPEC_DEFINE_PASSES(192)
}  // namespace pspec
