// sil_batch_k_u8.cu -- the batch kernel's instances for SIL_U8, H/S unconstrained.
#include "sil_batch_kernel.cuh"

namespace sil {
template struct BatchKernels<SIL_U8, false>;
}  // namespace sil
