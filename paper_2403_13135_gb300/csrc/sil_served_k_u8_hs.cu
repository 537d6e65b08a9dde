// sil_served_k_u8_hs.cu -- the served kernel's instances for SIL_U8, H/S narrowed.
#include "sil_served_kernel.cuh"

namespace sil {
template struct ServedKernels<SIL_U8, true>;
}  // namespace sil
