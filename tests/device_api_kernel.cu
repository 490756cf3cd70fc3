// Test shim: a user kernel that advances each exported stream state with the
// single-stream functions of prand_device.h (one thread per stream), writing
// m outputs per stream, stream-major, and leaving the advanced states in place.
#include <cuda_runtime.h>

#include "prand_device.h"

template <typename S, uint32_t (*NEXT)(S *)>
__global__ void run(S *states, unsigned long long n, uint32_t *out, unsigned long long m)
{
    const unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    S s = states[j];
    for (unsigned long long i = 0; i < m; ++i) out[j * m + i] = NEXT(&s);
    states[j] = s;
}

template <typename S, uint32_t (*NEXT)(S *)>
static int launch(void *states, unsigned long long n, uint32_t *out, unsigned long long m)
{
    run<S, NEXT><<<(unsigned)((n + 63) / 64), 64>>>((S *)states, n, out, m);
    return cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}

extern "C" int dev_api_kernel(int gen, void *states, unsigned long long n, uint32_t *out, unsigned long long m)
{
    switch (gen) {
    case 0: return launch<prand_mt19937_state, prand_mt19937_next_u32>(states, n, out, m);
    case 1: return launch<prand_mrg32k3a_state, prand_mrg32k3a_next_u32>(states, n, out, m);
    case 2: return launch<prand_lfsr113_state, prand_lfsr113_next_u32>(states, n, out, m);
    case 3: return launch<prand_gm_state, prand_gm19_next_u32>(states, n, out, m);
    case 4: return launch<prand_gm_state, prand_gm29_next_u32>(states, n, out, m);
    case 5: return launch<prand_gm_state, prand_gm31_next_u32>(states, n, out, m);
    case 6: return launch<prand_gm_state, prand_gm55_next_u32>(states, n, out, m);
    case 7: return launch<prand_gm_state, prand_gm61_next_u32>(states, n, out, m);
    case 8: return launch<prand_gm_state, prand_gq58_1_next_u32>(states, n, out, m);
    case 9: return launch<prand_gm_state, prand_gq58_3_next_u32>(states, n, out, m);
    case 10: return launch<prand_gm_state, prand_gq58_4_next_u32>(states, n, out, m);
    default: return -1;
    }
}
