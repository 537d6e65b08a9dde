// sil_batch_k_u16.cu -- the batch kernel's instances for SIL_U16, H/S unconstrained.
#include "sil_batch_kernel.cuh"

namespace sil {
template struct BatchKernels<SIL_U16, false>;
}  // namespace sil
