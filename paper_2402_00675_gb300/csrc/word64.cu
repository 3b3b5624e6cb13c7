// 64-bit word kernels: instantiation and dispatch by variant.
#include "word_kernel.cuh"

namespace montgb {

cudaError_t launch_word64(int variant, Mode mode, const WordConst64& c, const void* x,
                          const void* y, void* out, size_t n, cudaStream_t s,
                          const LaunchShape& shape) {
  switch (variant) {
    case MONT_REDC: return launch_mode<Redc64>(mode, c, x, y, out, n, s, shape);
    case MONT_SIGNED: return launch_mode<Signed64>(mode, c, x, y, out, n, s, shape);
    case MONT_PLANTARD: return launch_mode<Plantard64>(mode, c, x, y, out, n, s, shape);
    case MONT_SIGNED_PLANTARD: return launch_mode<SignedPlantard64>(mode, c, x, y, out, n, s, shape);
    case MONT_SIGNED_PLANTARD2:
      return launch_mode<SignedPlantard2_64>(mode, c, x, y, out, n, s, shape);
  }
  return cudaErrorInvalidValue;
}

}  // namespace montgb
