// GQ58.4 instantiation of the torus-map ensemble kernels (see gm_impl.cuh).
#include "gm_impl.cuh"

namespace prand {
PRAND_GM_INSTANTIATE(PRAND_GQ58_4, gq58_4)
}  // namespace prand
