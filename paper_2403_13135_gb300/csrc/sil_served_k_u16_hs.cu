// sil_served_k_u16_hs.cu -- the served kernel's instances for SIL_U16, H/S narrowed.
#include "sil_served_kernel.cuh"

namespace sil {
template struct ServedKernels<SIL_U16, true>;
}  // namespace sil
