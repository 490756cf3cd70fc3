// GQ58.3 instantiation of the torus-map ensemble kernels (see gm_impl.cuh).
#include "gm_impl.cuh"

namespace prand {
PRAND_GM_INSTANTIATE(PRAND_GQ58_3, gq58_3)
}  // namespace prand
