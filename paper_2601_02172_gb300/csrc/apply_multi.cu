// Stiffness apply kernels of two interfaces (three phases, Sec. 4.2's coated sphere); the
// one-interface kernels are instantiated in apply.cu.
#include "apply_kernels.cuh"

namespace xfft {

XFFT_APPLY_INST_NPH(, float, 3)
XFFT_APPLY_INST_NPH(, double, 3)
XFFT_APPLY_INST_NPH(, dw, 3)

}  // namespace xfft
