// sil_label_k_u8_hs.cu -- the single-request kernels for SIL_U8, H/S narrowed.
#include "sil_label_kernel.cuh"

namespace sil {
template struct LabelKernels<SIL_U8, true>;
}  // namespace sil
