// sil_label_k_u16_hs.cu -- the single-request kernels for SIL_U16, H/S narrowed.
#include "sil_label_kernel.cuh"

namespace sil {
template struct LabelKernels<SIL_U16, true>;
}  // namespace sil
