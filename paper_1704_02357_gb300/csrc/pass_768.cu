// Transform passes instantiated for mesh sides: 768.
#include "k_fft_kernels.cuh"

namespace pspec {
PSPEC_DEFINE_PASSES(768)
}  // namespace pspec
