// sil_served_k_u16.cu -- the served kernel's instances for SIL_U16, H/S unconstrained.
#include "sil_served_kernel.cuh"

namespace sil {
template struct ServedKernels<SIL_U16, false>;
}  // namespace sil
