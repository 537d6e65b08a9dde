// sil_batch_k_u8_hs.cu -- the batch kernel's instances for SIL_U8, H/S narrowed.
#include "sil_batch_kernel.cuh"

namespace sil {
template struct BatchKernels<SIL_U8, true>;
}  // namespace sil
