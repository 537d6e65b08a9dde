// sil_label_k_u16.cu -- the single-request kernels for SIL_U16, H/S unconstrained.
#include "sil_label_kernel.cuh"

namespace sil {
template struct LabelKernels<SIL_U16, false>;
}  // namespace sil
