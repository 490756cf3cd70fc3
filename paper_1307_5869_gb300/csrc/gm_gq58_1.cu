// GQ58.1 instantiation of the torus-map ensemble kernels (see gm_impl.cuh).
#include "gm_impl.cuh"

namespace prand {
PRAND_GM_INSTANTIATE(PRAND_GQ58_1, gq58_1)
}  // namespace prand
