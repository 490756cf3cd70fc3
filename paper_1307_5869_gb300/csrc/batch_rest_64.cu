// The rest-of-generators build of the batched persistent kernel with 64
// threads per block, in its 128- and 256-byte staged-row forms (a translation
// unit of its own, so the builds compile in parallel).
#include "batch_kernel.cuh"

namespace prand {

int rest_blocks_per_sm_64(bool row256)
{
    int bps = 0;
    const cudaError_t e = row256
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel<kModeRest, 64, 256>, 64, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel<kModeRest, 64, 128>, 64, 0);
    return (e == cudaSuccess && bps >= 1) ? bps : 1;
}

void rest_launch_64(bool row256, unsigned grid, cudaStream_t st, const BatchTile *tiles, uint32_t ntiles,
                    uint32_t *counter, const BatchCtx &ctx)
{
    if (row256) batch_kernel<kModeRest, 64, 256><<<grid, 64, 0, st>>>(tiles, ntiles, counter, ctx);
    else batch_kernel<kModeRest, 64, 128><<<grid, 64, 0, st>>>(tiles, ntiles, counter, ctx);
}

}  // namespace prand
