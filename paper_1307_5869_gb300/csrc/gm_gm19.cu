// GM19 instantiation of the torus-map ensemble kernels (see gm_impl.cuh).
#include "gm_impl.cuh"

namespace prand {
PRAND_GM_INSTANTIATE(PRAND_GM19, gm19)
}  // namespace prand
