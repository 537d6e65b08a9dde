// sil_label_k_u8.cu -- the single-request kernels for SIL_U8, H/S unconstrained.
#include "sil_label_kernel.cuh"

namespace sil {
template struct LabelKernels<SIL_U8, false>;
}  // namespace sil
