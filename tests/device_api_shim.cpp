// Test shim: the single-stream functions of prand_device.h compiled for the
// host, driven through a C entry point.
#include <string.h>

#include "prand_device.h"

extern "C" int dev_api_run(int gen, void *state, int kind, void *out, unsigned long long n)
{
    for (unsigned long long i = 0; i < n; ++i) {
        uint32_t u;
        switch (gen) {
        case 0: u = prand_mt19937_next_u32((prand_mt19937_state *)state); break;
        case 1: u = prand_mrg32k3a_next_u32((prand_mrg32k3a_state *)state); break;
        case 2: u = prand_lfsr113_next_u32((prand_lfsr113_state *)state); break;
        case 3: u = prand_gm19_next_u32((prand_gm_state *)state); break;
        case 4: u = prand_gm29_next_u32((prand_gm_state *)state); break;
        case 5: u = prand_gm31_next_u32((prand_gm_state *)state); break;
        case 6: u = prand_gm55_next_u32((prand_gm_state *)state); break;
        case 7: u = prand_gm61_next_u32((prand_gm_state *)state); break;
        case 8: u = prand_gq58_1_next_u32((prand_gm_state *)state); break;
        case 9: u = prand_gq58_3_next_u32((prand_gm_state *)state); break;
        case 10: u = prand_gq58_4_next_u32((prand_gm_state *)state); break;
        default: return -1;
        }
        if (kind == 0) ((uint32_t *)out)[i] = u;
        else if (kind == 1) ((float *)out)[i] = prand_u32_to_f32(u);
        else ((double *)out)[i] = gen == 1 ? prand_mrg32k3a_to_f64(u) : prand_u32_to_f64(u);
    }
    return 0;
}
