// sil_served_k_u8.cu -- the served kernel's instances for SIL_U8, H/S unconstrained.
#include "sil_served_kernel.cuh"

namespace sil {
template struct ServedKernels<SIL_U8, false>;
}  // namespace sil
