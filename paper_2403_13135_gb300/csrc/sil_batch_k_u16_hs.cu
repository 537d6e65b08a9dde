// sil_batch_k_u16_hs.cu -- the batch kernel's instances for SIL_U16, H/S narrowed.
#include "sil_batch_kernel.cuh"

namespace sil {
template struct BatchKernels<SIL_U16, true>;
}  // namespace sil
