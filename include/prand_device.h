/* Single-stream generation inside user code (host or device): the paper's
 * single-threaded interface (Sec. 7.3, rng_generate_ and
 * rng_generate_uniform_float_), one state per stream, one output per call.
 *
 * Header-only C++.  Under nvcc every function is __host__ __device__, so a
 * user kernel can give each thread its own stream; a host compiler gets plain
 * inline functions.  The states are exchanged with a handle by
 * prand_export_states / prand_import_states (prand.h), one struct per stream
 * in the layout below; the sequences are exactly those of prand_generate_*:
 *   u32: the generator's 32-bit output (MRG32K3A: z in [1, m1]);
 *   f32: (u >> 8) 2^-24 in [0, 1);
 *   f64: u 2^-32 in [0, 1); MRG32K3A: z RN(1 / (m1 + 1)) in (0, 1).
 * These functions favour plainness over speed (one stream at a time; a GM/GQ
 * output word steps all of its points); the library's kernels are the fast
 * path for filling arrays.
 */
#ifndef PRAND_DEVICE_H
#define PRAND_DEVICE_H

#include <stdint.h>

#if defined(__CUDACC__)
#define PRAND_HD __host__ __device__ __forceinline__
#else
#define PRAND_HD inline
#endif

/* ------------------------------------------------------------ state layouts */

/* MT19937 (Sec. 5.4): the current 624-word block and the index of the next
 * word to temper (624: the block is used up and is twisted before the next
 * output). */
typedef struct { uint32_t mt[624]; uint32_t idx; } prand_mt19937_state;

/* MRG32K3A (Sec. 5.2): x = (x_n, x_{n-1}, x_{n-2}) mod m1, y likewise mod m2. */
typedef struct { uint32_t x[3]; uint32_t y[3]; } prand_mrg32k3a_state;

/* LFSR113 (Sec. 5.3): the four component words. */
typedef struct { uint32_t z[4]; } prand_lfsr113_state;

/* GM / GQ ensembles (Sec. 5.1): (x^(n-1), x^(n)) of each point, x mod g; the
 * first s entries are used (s = 32, 8 or 12 points per output word). */
typedef struct { uint64_t x_prev[32]; uint64_t x[32]; } prand_gm_state;

/* ------------------------------------------------------------ float maps */

PRAND_HD float prand_u32_to_f32(uint32_t u) { return (float)(u >> 8) * 0x1p-24f; }
PRAND_HD double prand_u32_to_f64(uint32_t u) { return (double)u * 0x1p-32; }
PRAND_HD double prand_mrg32k3a_to_f64(uint32_t z)
{
#if defined(__CUDA_ARCH__)
    return __dmul_rn((double)z, 1.0 / 4294967088.0);
#else
    return (double)z * (1.0 / 4294967088.0);
#endif
}

/* ------------------------------------------------------------ MT19937 */

PRAND_HD uint32_t prand_mt19937_next_u32(prand_mt19937_state *s)
{
    if (s->idx >= 624) {
        for (int k = 0; k < 624; ++k) {
            const uint32_t y = (s->mt[k] & 0x80000000u) | (s->mt[(k + 1) % 624] & 0x7FFFFFFFu);
            s->mt[k] = s->mt[(k + 397) % 624] ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
        }
        s->idx = 0;
    }
    uint32_t y = s->mt[s->idx++];
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

/* ------------------------------------------------------------ MRG32K3A */

PRAND_HD uint32_t prand_mrg32k3a_next_u32(prand_mrg32k3a_state *s)
{
    const uint64_t m1 = 4294967087ull, m2 = 4294944443ull;
    /* x_{n+1} = 1403580 x_{n-1} - 810728 x_{n-2} (mod m1), kept non-negative */
    const uint64_t xn = (1403580ull * s->x[1] % m1 + 810728ull * (m1 - s->x[2]) % m1) % m1;
    /* y_{n+1} = 527612 y_n - 1370589 y_{n-2} (mod m2) */
    const uint64_t yn = (527612ull * s->y[0] % m2 + 1370589ull * (m2 - s->y[2]) % m2) % m2;
    s->x[2] = s->x[1]; s->x[1] = s->x[0]; s->x[0] = (uint32_t)xn;
    s->y[2] = s->y[1]; s->y[1] = s->y[0]; s->y[0] = (uint32_t)yn;
    return (uint32_t)(xn > yn ? xn - yn : xn + m1 - yn);  /* (x - y) mod m1, 0 -> m1 */
}

/* ------------------------------------------------------------ LFSR113 */

PRAND_HD uint32_t prand_lfsr113_next_u32(prand_lfsr113_state *s)
{
    /* component (p, q, s): (31, 6, 18), (29, 2, 2), (28, 13, 7), (25, 3, 13) */
    s->z[0] = ((s->z[0] & 0xFFFFFFFEu) << 18) ^ (((s->z[0] << 6) ^ s->z[0]) >> 13);
    s->z[1] = ((s->z[1] & 0xFFFFFFF8u) << 2) ^ (((s->z[1] << 2) ^ s->z[1]) >> 27);
    s->z[2] = ((s->z[2] & 0xFFFFFFF0u) << 7) ^ (((s->z[2] << 13) ^ s->z[2]) >> 21);
    s->z[3] = ((s->z[3] & 0xFFFFFF80u) << 13) ^ (((s->z[3] << 3) ^ s->z[3]) >> 12);
    return s->z[0] ^ s->z[1] ^ s->z[2] ^ s->z[3];
}

/* ------------------------------------------------------------ GM / GQ */

/* a b mod m for a, b < m < 2^62, by a 128-bit product */
PRAND_HD uint64_t prand_mulmod64(uint64_t a, uint64_t b, uint64_t m)
{
#if defined(__CUDA_ARCH__)
    /* long division of the 128-bit product, one bit at a time */
    uint64_t hi = __umul64hi(a, b), lo = a * b, r = 0;
    for (int i = 127; i >= 0; --i) {
        const uint64_t bit = i >= 64 ? (hi >> (i - 64)) & 1u : (lo >> i) & 1u;
        r = (r << 1) | bit;
        if (r >= m) r -= m;
    }
    return r;
#else
    return (uint64_t)((unsigned __int128)a * b % m);
#endif
}

/* One output word of an ensemble: every point takes one step of eq. (rec1),
 * x' = k x - q x_prev (mod g), and point i contributes floor(2^v x' / g) at bit
 * v i (bits at 32 and above are dropped). */
PRAND_HD uint32_t prand_gm_next_u32_generic(prand_gm_state *st, uint64_t k, uint64_t q, uint64_t g, int v, int s)
{
    uint32_t w = 0;
    for (int i = 0; i < s; ++i) {
        const uint64_t kx = prand_mulmod64(k % g, st->x[i], g);
        const uint64_t qx = prand_mulmod64(q % g, st->x_prev[i], g);
        const uint64_t xn = kx >= qx ? kx - qx : kx + (g - qx);
        st->x_prev[i] = st->x[i];
        st->x[i] = xn;
        /* strip index floor(2^v xn / g) < 2^v, without overflow: compare with
         * the strip boundaries ceil(j g / 2^v) */
        uint32_t strip = 0;
        for (int j = 1; j < (1 << v); ++j) {
            const uint64_t bound = (uint64_t)(((unsigned __int128)g * (unsigned)j + ((1u << v) - 1)) >> v);
            if (xn >= bound) strip = (uint32_t)j;
        }
        if (v * i < 32) w |= strip << (v * i);
    }
    return w;
}

/* Parameters of Table 2 (k, q, g, v) and the points per word s. */
#define PRAND_GM_NEXT(NAME, K, Q, G, V, S)                                                                \
    PRAND_HD uint32_t prand_##NAME##_next_u32(prand_gm_state *st)                                      \
    {                                                                                                  \
        return prand_gm_next_u32_generic(st, (K), (Q), (G), (V), (S));                                  \
    }
PRAND_GM_NEXT(gm19, 15ull, 28ull, (1ull << 19) - 1, 1, 32)
PRAND_GM_NEXT(gm29, 4ull, 2ull, (1ull << 29) - 3, 1, 32)
PRAND_GM_NEXT(gm31, 11ull, 14ull, (1ull << 31) - 1, 1, 32)
PRAND_GM_NEXT(gm55, 256ull, 176ull, 16ull * ((1ull << 51) - 129), 4, 8)
PRAND_GM_NEXT(gm61, 24ull, 74ull, (1ull << 61) - 1, 1, 32)
PRAND_GM_NEXT(gq58_1, 8ull, 48ull, (1ull << 29) * ((1ull << 29) - 3), 1, 32)
PRAND_GM_NEXT(gq58_3, 8ull, 48ull, (1ull << 29) * ((1ull << 29) - 3), 3, 12)
PRAND_GM_NEXT(gq58_4, 8ull, 48ull, (1ull << 29) * ((1ull << 29) - 3), 4, 8)
#undef PRAND_GM_NEXT

#endif /* PRAND_DEVICE_H */
