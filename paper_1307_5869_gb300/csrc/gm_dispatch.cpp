// Dispatch of the GM/GQ entry points to the per-generator translation units,
// and the host copy of the Table 2 / Table 4 parameters.
#include "prand_internal.h"

namespace prand {

prand_status_t gm19_table(uint64_t *, cudaStream_t);
prand_status_t gm19_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm19_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm19_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gm19_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gm29_table(uint64_t *, cudaStream_t);
prand_status_t gm29_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm29_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm29_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gm29_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gm31_table(uint64_t *, cudaStream_t);
prand_status_t gm31_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm31_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm31_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gm31_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gm55_table(uint64_t *, cudaStream_t);
prand_status_t gm55_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm55_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm55_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gm55_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gm61_table(uint64_t *, cudaStream_t);
prand_status_t gm61_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm61_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gm61_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gm61_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gq58_1_table(uint64_t *, cudaStream_t);
prand_status_t gq58_1_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gq58_1_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gq58_1_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gq58_1_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gq58_3_table(uint64_t *, cudaStream_t);
prand_status_t gq58_3_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gq58_3_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gq58_3_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gq58_3_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);
prand_status_t gq58_4_table(uint64_t *, cudaStream_t);
prand_status_t gq58_4_seed(const uint64_t *, uint64_t *, uint64_t, const Variant &, cudaStream_t);
prand_status_t gq58_4_init(const uint64_t *, const uint64_t *, uint64_t *, uint64_t, uint64_t, const Variant &, cudaStream_t);
prand_status_t gq58_4_skip(const uint64_t *, uint64_t *, uint64_t, const U256 &, cudaStream_t);
prand_status_t gq58_4_gen(const uint64_t *, uint64_t *, uint64_t *, StreamRange &, void *, int, uint64_t, cudaStream_t);

static const GmParams kGmHost[8] = {
    { 15, 28, (1ull << 19) - 1, 0, 1, 32, 32, P19, 6000000ull, 1000ull },
    { 4, 2, (1ull << 29) - 3, 0, 1, 32, 32, P29, 80000000ull, 100000000ull },
    { 11, 14, (1ull << 31) - 1, 0, 1, 32, 32, P31, 80000000ull, 1000000000ull },
    { 256, 176, (1ull << 51) - 129, 4, 4, 8, 1, P51, 10000000000ull, 1000000000000000000ull },
    { 24, 74, (1ull << 61) - 1, 0, 1, 32, 32, P61, 10000000000ull, 18000000000000000000ull },
    { 8, 48, (1ull << 29) - 3, 29, 1, 32, 32, P29, 80000000ull, 100000000ull },
    { 8, 48, (1ull << 29) - 3, 29, 3, 12, 1, P29, 80000000ull, 200000000ull },
    { 8, 48, (1ull << 29) - 3, 29, 4, 8, 1, P29, 80000000ull, 300000000ull },
};



const GmParams &gm_params(int gen) { return kGmHost[gen - PRAND_GM19]; }

prand_status_t gm_build_table(int gen, uint64_t *tab, cudaStream_t st)
{
    switch (gen) {
    case PRAND_GM19: return gm19_table(tab, st);
    case PRAND_GM29: return gm29_table(tab, st);
    case PRAND_GM31: return gm31_table(tab, st);
    case PRAND_GM55: return gm55_table(tab, st);
    case PRAND_GM61: return gm61_table(tab, st);
    case PRAND_GQ58_1: return gq58_1_table(tab, st);
    case PRAND_GQ58_3: return gq58_3_table(tab, st);
    case PRAND_GQ58_4: return gq58_4_table(tab, st);
    default: return PRAND_ERR_ARG;
    }
}

prand_status_t gm_seed(int gen, const DevTables *T, uint64_t seed, const Variant &V, void *d_base, cudaStream_t st)
{
    const uint64_t *tab = T->gm[gen - PRAND_GM19];
    uint64_t *base = (uint64_t *)d_base;
    switch (gen) {
    case PRAND_GM19: return gm19_seed(tab, base, seed, V, st);
    case PRAND_GM29: return gm29_seed(tab, base, seed, V, st);
    case PRAND_GM31: return gm31_seed(tab, base, seed, V, st);
    case PRAND_GM55: return gm55_seed(tab, base, seed, V, st);
    case PRAND_GM61: return gm61_seed(tab, base, seed, V, st);
    case PRAND_GQ58_1: return gq58_1_seed(tab, base, seed, V, st);
    case PRAND_GQ58_3: return gq58_3_seed(tab, base, seed, V, st);
    case PRAND_GQ58_4: return gq58_4_seed(tab, base, seed, V, st);
    default: return PRAND_ERR_ARG;
    }
}

prand_status_t gm_init(int gen, const DevTables *T, const void *d_base, void *d_state, uint64_t first, uint64_t n,
                       const Variant &V, cudaStream_t st)
{
    const uint64_t *tab = T->gm[gen - PRAND_GM19];
    const uint64_t *base = (const uint64_t *)d_base;
    uint64_t *state = (uint64_t *)d_state;
    switch (gen) {
    case PRAND_GM19: return gm19_init(tab, base, state, first, n, V, st);
    case PRAND_GM29: return gm29_init(tab, base, state, first, n, V, st);
    case PRAND_GM31: return gm31_init(tab, base, state, first, n, V, st);
    case PRAND_GM55: return gm55_init(tab, base, state, first, n, V, st);
    case PRAND_GM61: return gm61_init(tab, base, state, first, n, V, st);
    case PRAND_GQ58_1: return gq58_1_init(tab, base, state, first, n, V, st);
    case PRAND_GQ58_3: return gq58_3_init(tab, base, state, first, n, V, st);
    case PRAND_GQ58_4: return gq58_4_init(tab, base, state, first, n, V, st);
    default: return PRAND_ERR_ARG;
    }
}

prand_status_t gm_skip(int gen, const DevTables *T, void *d_state, uint64_t n, const U256 &off, cudaStream_t st)
{
    const uint64_t *tab = T->gm[gen - PRAND_GM19];
    uint64_t *state = (uint64_t *)d_state;
    switch (gen) {
    case PRAND_GM19: return gm19_skip(tab, state, n, off, st);
    case PRAND_GM29: return gm29_skip(tab, state, n, off, st);
    case PRAND_GM31: return gm31_skip(tab, state, n, off, st);
    case PRAND_GM55: return gm55_skip(tab, state, n, off, st);
    case PRAND_GM61: return gm61_skip(tab, state, n, off, st);
    case PRAND_GQ58_1: return gq58_1_skip(tab, state, n, off, st);
    case PRAND_GQ58_3: return gq58_3_skip(tab, state, n, off, st);
    case PRAND_GQ58_4: return gq58_4_skip(tab, state, n, off, st);
    default: return PRAND_ERR_ARG;
    }
}

prand_status_t gm_gen(int gen, const DevTables *T, void *d_state, void *d_spare, StreamRange &R, void *out, int dtype,
                      uint64_t nper, cudaStream_t st)
{
    const uint64_t *tab = T->gm[gen - PRAND_GM19];
    uint64_t *s = (uint64_t *)d_state, *sp = (uint64_t *)d_spare;
    switch (gen) {
    case PRAND_GM19: return gm19_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GM29: return gm29_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GM31: return gm31_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GM55: return gm55_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GM61: return gm61_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GQ58_1: return gq58_1_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GQ58_3: return gq58_3_gen(tab, s, sp, R, out, dtype, nper, st);
    case PRAND_GQ58_4: return gq58_4_gen(tab, s, sp, R, out, dtype, nper, st);
    default: return PRAND_ERR_ARG;
    }
}

}  // namespace prand
