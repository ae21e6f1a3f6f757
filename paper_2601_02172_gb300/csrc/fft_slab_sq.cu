// Slab-path launchers for the y-z plane sizes below 128 (kernels in fft_slab.cuh).
#include "fft_slab.cuh"

namespace xfft {
namespace slab {
XFFT_SLAB_SMALL(XFFT_SLAB_INST)
}  // namespace slab
}  // namespace xfft
