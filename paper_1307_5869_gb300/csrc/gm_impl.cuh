// GM19, GM29, GM31, GM55, GM61, GQ58.1, GQ58.3, GQ58.4: ensembles of s
// two-dimensional torus maps x^(n) = k x^(n-1) - q x^(n-2) (mod g) (Sec. 5.1,
// eq. (rec1), parameters of Table 2).
//
// Two GPU layouts, by the bits per point v:
//  * v = 1 (GM19, GM29, GM31, GM61, GQ58.1; 32 points per word): a warp runs
//    one stream, one torus point per lane; each lane does one recurrence step
//    per output word and the word is one warp ballot (lane i <-> bit i).  The
//    warp then hands word t to lane (t / 4) mod 32, which emits four words at
//    a time as one 16-byte store.
//  * v = 3, 4 (GQ58.3: 12 points; GM55, GQ58.4: 8 points): one thread runs
//    one stream section with all of its points in registers; each point's
//    strip is extracted from one 64-bit sum by a funnel shift and placed in the
//    word by one logic operation, so no lane waits on another.  Rows leave
//    through the staged 128-byte row stores of the thread-per-stream
//    generators.
//
// Arithmetic is exact on z = x / 2^t modulo the prime p (g = 2^t p; for GM55
// and GQ58.x, k and q are even, so states kept on multiples of 2^t stay there
// and z follows the same recurrence mod p), in 32-bit limbs written out in
// inline PTX: the products are 32x32 -> 32 or 64-bit multiply-adds and each
// step folds once (lazy residues, below).  The state is stored as x = 2^t z,
// (x^(n-1), x^(n)) per point.
//
// Readings (the paper prints only k, q, g, v): s = 32 points for v = 1, 8 for
// v = 4, 12 for GQ58.3 (Table 5's threads per section); point i contributes
// floor(2^v x_i / g) at bit v*i (truncated to 32 bits); point i of the base
// ensemble is the base pair advanced by i * D, D = nmax * L (Table 4).
#pragma once
#include <type_traits>
#include <utility>

#include "devcommon.cuh"

namespace prand {

template <int GEN>
struct GmT;
// k, q, p, t, v, s, lanes per stream (32: lane per point; 1: thread per
// stream), prime kind, L, nmax
#define PRAND_GM_TRAITS(GEN, K, Q, PP, T, V, S, LANES, KIND, L, NMAX)                                   \
    template <>                                                                                       \
    struct GmT<GEN> {                                                                                 \
        static constexpr uint64_t k = K, q = Q, p = PP, L_ = L, nmax = NMAX;                            \
        static constexpr int t = T, v = V, s = S, lanes = LANES, kind = KIND;                          \
    };
PRAND_GM_TRAITS(PRAND_GM19, 15, 28, (1ull << 19) - 1, 0, 1, 32, 32, P19, 6000000ull, 1000ull)
PRAND_GM_TRAITS(PRAND_GM29, 4, 2, (1ull << 29) - 3, 0, 1, 32, 32, P29, 80000000ull, 100000000ull)
PRAND_GM_TRAITS(PRAND_GM31, 11, 14, (1ull << 31) - 1, 0, 1, 32, 32, P31, 80000000ull, 1000000000ull)
PRAND_GM_TRAITS(PRAND_GM55, 256, 176, (1ull << 51) - 129, 4, 4, 8, 1, P51, 10000000000ull, 1000000000000000000ull)
PRAND_GM_TRAITS(PRAND_GM61, 24, 74, (1ull << 61) - 1, 0, 1, 32, 32, P61, 10000000000ull, 18000000000000000000ull)
PRAND_GM_TRAITS(PRAND_GQ58_1, 8, 48, (1ull << 29) - 3, 29, 1, 32, 32, P29, 80000000ull, 100000000ull)
PRAND_GM_TRAITS(PRAND_GQ58_3, 8, 48, (1ull << 29) - 3, 29, 3, 12, 1, P29, 80000000ull, 200000000ull)
PRAND_GM_TRAITS(PRAND_GQ58_4, 8, 48, (1ull << 29) - 3, 29, 4, 8, 1, P29, 80000000ull, 300000000ull)
#undef PRAND_GM_TRAITS

// Register type of a residue during generation: 32 bits when p < 2^32.
template <int GEN>
using GmZ = typename std::conditional<(GmT<GEN>::p < (1ull << 32)), uint32_t, uint64_t>::type;

// ----------------------------------------------------------------- one step
// z' = k z - q z_prev (mod p) with lazy residues: between steps z stays in
// [0, p + slack) (slack below), so a step needs one fold and no final
// comparison.  Every fold is S - h p (h = the bits of S above the prime's
// width), one multiply-add.  canon() returns the residue in [0, p); all lazy
// ranges are below 2p.
template <int GEN>
__device__ __forceinline__ uint64_t gm_canon(uint64_t z)
{
    constexpr uint64_t p = GmT<GEN>::p;
    return z >= p ? z - p : z;
}

template <int GEN>
__device__ __forceinline__ GmZ<GEN> gm_step(GmZ<GEN> zc, GmZ<GEN> zp);

// p = 2^19 - 1; lazy z < 2^19 + 72.  S = 15 z + 28 (2p - y) = 15 z + 56 p - 28 y
// lies in (0, 2^26); h = S >> 19 < 72 and S - h p = (S mod 2^19) + h.
template <>
__device__ __forceinline__ uint32_t gm_step<PRAND_GM19>(uint32_t z, uint32_t y)
{
    uint32_t r;
    asm("{\n\t"
        ".reg .u32 a, h;\n\t"
        "mad.lo.u32 a, %2, 0xFFFFFFE4, 29360072;\n\t"   // 56 p - 28 y
        "mad.lo.u32 a, %1, 15, a;\n\t"
        "shr.u32 h, a, 19;\n\t"
        "mad.lo.u32 %0, h, 0xFFF80001, a;\n\t"           // S - h (2^19 - 1)
        "}"
        : "=r"(r) : "r"(z), "r"(y));
    return r;
}
// p = 2^29 - 3; lazy z < 2^29 + 24.  S = 4 z + 3 p - 2 y lies in (2^29 - 57,
// 2^32); h = S >> 29 <= 7 and S - h p = (S mod 2^29) + 3 h.
template <>
__device__ __forceinline__ uint32_t gm_step<PRAND_GM29>(uint32_t z, uint32_t y)
{
    uint32_t r;
    asm("{\n\t"
        ".reg .u32 a, h;\n\t"
        "mad.lo.u32 a, %2, 0xFFFFFFFE, 1610612727;\n\t"  // 3 p - 2 y
        "mad.lo.u32 a, %1, 4, a;\n\t"
        "shr.u32 h, a, 29;\n\t"
        "mad.lo.u32 %0, h, 0xE0000003, a;\n\t"           // S - h (2^29 - 3)
        "}"
        : "=r"(r) : "r"(z), "r"(y));
    return r;
}
// p = 2^31 - 1; lazy z < 2^31 + 40.  S = 11 z + 14 (2p - y) < 40 * 2^31 by two
// wide multiply-adds; h = S >> 31 < 40 and S - h p = (S mod 2^31) + h, computed
// in the low word (the true value is below 2^32).
template <>
__device__ __forceinline__ uint32_t gm_step<PRAND_GM31>(uint32_t z, uint32_t y)
{
    uint32_t r;
    asm("{\n\t"
        ".reg .u32 t, lo, hi, h;\n\t"
        ".reg .u64 T, S;\n\t"
        "sub.u32 t, 0xFFFFFFFE, %2;\n\t"                 // 2 p - y
        "mul.wide.u32 T, t, 14;\n\t"
        "mad.wide.u32 S, %1, 11, T;\n\t"
        "mov.b64 {lo, hi}, S;\n\t"
        "shf.r.wrap.b32 h, lo, hi, 31;\n\t"
        "mad.lo.u32 %0, h, 0x80000001, lo;\n\t"          // S - h (2^31 - 1)
        "}"
        : "=r"(r) : "r"(z), "r"(y));
    return r;
}
// p = 2^29 - 3 (GQ58.x, z = x / 2^29); lazy z < 2^29 + 312.  S = 8 z + 48 (2p -
// y) < 2^36; h = S >> 29 <= 104 and S - h p = (S mod 2^29) + 3 h.
__device__ __forceinline__ uint32_t gq58_step(uint32_t z, uint32_t y)
{
    uint32_t r;
    asm("{\n\t"
        ".reg .u32 t, lo, hi, h;\n\t"
        ".reg .u64 T, S;\n\t"
        "sub.u32 t, 1073741818, %2;\n\t"                 // 2 p - y
        "mul.wide.u32 T, t, 48;\n\t"
        "mad.wide.u32 S, %1, 8, T;\n\t"
        "mov.b64 {lo, hi}, S;\n\t"
        "shf.r.wrap.b32 h, lo, hi, 29;\n\t"
        "mad.lo.u32 %0, h, 0xE0000003, lo;\n\t"          // S - h (2^29 - 3)
        "}"
        : "=r"(r) : "r"(z), "r"(y));
    return r;
}
template <>
__device__ __forceinline__ uint32_t gm_step<PRAND_GQ58_1>(uint32_t z, uint32_t y) { return gq58_step(z, y); }
template <>
__device__ __forceinline__ uint32_t gm_step<PRAND_GQ58_3>(uint32_t z, uint32_t y) { return gq58_step(z, y); }
template <>
__device__ __forceinline__ uint32_t gm_step<PRAND_GQ58_4>(uint32_t z, uint32_t y) { return gq58_step(z, y); }
// p = 2^51 - 129; lazy z < 2^51 + 129 * 2^10.  In 32-bit limbs: t = 2p - y
// (< 2^52), S = 256 z + 176 t < 2^61 (low limbs by two wide multiply-adds, the
// high word by two more), h = S >> 51 < 2^10, S - h p = (S mod 2^51) + 129 h.
template <>
__device__ __forceinline__ uint64_t gm_step<PRAND_GM55>(uint64_t z, uint64_t y)
{
    uint32_t r0, r1;
    asm("{\n\t"
        ".reg .u32 t0, t1, a0, a1, s1, h;\n\t"
        ".reg .u64 T, U;\n\t"
        "sub.cc.u32 t0, 0xFFFFFEFE, %2;\n\t"             // 2 p = 2^52 - 258
        "subc.u32 t1, 0x000FFFFF, %3;\n\t"
        "mul.wide.u32 T, t0, 176;\n\t"
        "mad.wide.u32 U, %4, 256, T;\n\t"                // < 2^41
        "mov.b64 {a0, a1}, U;\n\t"
        "mad.lo.u32 a1, t1, 176, a1;\n\t"
        "mad.lo.u32 s1, %5, 256, a1;\n\t"                // high word of S, < 2^29
        "shr.u32 h, s1, 19;\n\t"
        "mad.lo.cc.u32 %0, h, 129, a0;\n\t"
        "and.b32 s1, s1, 0x7FFFF;\n\t"
        "addc.u32 %1, s1, 0;\n\t"
        "}"
        : "=r"(r0), "=r"(r1)
        : "r"((uint32_t)y), "r"((uint32_t)(y >> 32)), "r"((uint32_t)z), "r"((uint32_t)(z >> 32)));
    return ((uint64_t)r1 << 32) | r0;
}
// p = 2^61 - 1.  Generation runs on u = (2 z mod p) + 1 rather than on z.
// Doubling modulo a Mersenne prime rotates the 61-bit residue left by one bit,
// so bit 60 of z -- the output bit floor(2 z / p) -- lands on bit 0; since the
// map is linear the doubled values obey the same recurrence, and the offset
// turns it into u' = 24 u - 74 u_prev + 51 (mod p).  Residues stay lazy in
// [1, 2^61 + 2^40): a value u >= 2^61 stands for u - p, whose bit 0 is the
// complement of u's, so the output bit is XNOR(bit 0 of u, bit 61 of u) --
// one logic operation instead of a 64-bit range test.
__device__ __forceinline__ uint64_t gm61_enter(uint64_t z)  // z lazy (< 2^61 + 256) -> u
{
    constexpr uint64_t p = (1ull << 61) - 1;
    const uint64_t c = z >= p ? z - p : z;
    return (((c << 1) & p) | (c >> 60)) + 1;
}
__device__ __forceinline__ uint64_t gm61_leave(uint64_t u)  // u (< 2p) -> canonical z
{
    constexpr uint64_t p = (1ull << 61) - 1;
    uint64_t w = u - 1;
    if (w >= p) w -= p;
    return (w >> 1) | ((w & 1) << 60);
}
// One step on (u, u_prev) in 32-bit limbs.  With t = C - u_prev, where
// C = 0x23E45306EB3E4530 > 2^61 + 2^40 and 74 C = 51 (mod p),
// S = 24 u + 74 t = u' (mod p).  A = 74 t0 + 24 u0 (< 2^39) and
// B = 74 t1 + 24 u1 (< 2^37) are independent 64-bit multiply-adds, so
// S = A + 2^32 B; with h = B >> 29 and m = B mod 2^29, 2^61 = 1 (mod p) gives
// S = A.lo + h + 2^32 (m + A.hi) (mod p), which is below 2^61 + 2^40 and at
// least 1 (it is 0 only if S = 0, and S > 0).  Adding A.hi after the fold,
// rather than into B, keeps every 64-bit accumulator a product's own register
// pair.  Returns the output bit of the new value.
__device__ __forceinline__ bool gm61_step(uint64_t &uc, uint64_t &up)
{
    const uint32_t u0 = (uint32_t)uc, u1 = (uint32_t)(uc >> 32);
    const uint32_t v0 = (uint32_t)up, v1 = (uint32_t)(up >> 32);
    uint32_t r0, r1;
    asm("{\n\t"
        ".reg .u32 t0, t1, a0, a1, b0, b1, h, m;\n\t"
        ".reg .u64 A, B, T, U;\n\t"
        "sub.cc.u32 t0, 0xEB3E4530, %2;\n\t"
        "subc.u32 t1, 0x23E45306, %3;\n\t"
        "mul.wide.u32 T, t0, 74;\n\t"
        "mad.wide.u32 A, %4, 24, T;\n\t"
        "mul.wide.u32 U, t1, 74;\n\t"
        "mad.wide.u32 B, %5, 24, U;\n\t"
        "mov.b64 {a0, a1}, A;\n\t"
        "mov.b64 {b0, b1}, B;\n\t"
        "shf.r.wrap.b32 h, b0, b1, 29;\n\t"
        "mad.lo.u32 m, h, 0xE0000000, b0;\n\t"
        "add.cc.u32 %0, a0, h;\n\t"
        "addc.u32 %1, m, a1;\n\t"
        "}"
        : "=r"(r0), "=r"(r1)
        : "r"(v0), "r"(v1), "r"(u0), "r"(u1));
    up = uc;
    uc = ((uint64_t)r1 << 32) | r0;
    return (((r0 << 29) ^ ~r1) & 0x20000000u) != 0;
}

// ----------------------------------------------------------------- strips
// floor(2^v z / p) of the canonical residue = floor(2^v x / g): the strip of the
// torus the point lies in, evaluated on the lazy value z.
template <int GEN>
__device__ __forceinline__ bool gm_strip1(uint32_t z)  // v = 1, p < 2^32: canonical z in [(p+1)/2, p)
{
    using P = GmT<GEN>;
    constexpr uint32_t half = (uint32_t)((P::p + 1) / 2);
    return z - half < (uint32_t)(P::p - half);
}

// v = 3, 4: the strip of point I placed at bit v I of the word w.  For
// p = 2^b - c, 2^v z = q0 2^b + r0 with q0 = z >> (b - v), and
// floor(2^v z / p) = q0 + [r0 + c q0 >= p] = (2^v z + c q0 + c) >> b (a
// 64-bit sum for GM55, a 32-bit one for p = 2^29 - 3); its low v bits are
// moved to bit v I by a shift and kept by a mask.  A lazy z in [p, p + slack) gives 2^v, whose
// low v bits are 0, the strip of z - p.  Bits beyond 31 are dropped (GQ58.3's
// point 10 keeps 2 of its 3 bits, point 11 none).
template <int GEN, int I>
__device__ __forceinline__ uint32_t gm_strip_insert(GmZ<GEN> z, uint32_t w)
{
    using P = GmT<GEN>;
    constexpr int v = P::v, pos = v * I;
    if constexpr (pos >= 32) {
        return w;
    } else if constexpr (P::kind == P51) {
        // p = 2^51 - 129, lazy z < 2^51 + 2^18: X = 16 z + 129 (q0 + 1) < 2^56;
        // the strip is bits 51..54 of X, i.e. bits 19..22 of its high word
        const uint32_t q0 = (uint32_t)(z >> 47);
        const uint64_t X = (z << 4) + (uint64_t)(129u * q0 + 129u);
        const uint32_t hi = (uint32_t)(X >> 32);
        const uint32_t x = pos <= 19 ? hi >> (19 - pos) : hi << (pos - 19);
        return (x & (15u << pos)) | w;
    } else {
        // p = 2^29 - 3, lazy z < 2^29 + 312: X = 2^v z + 3 (q0 + 1) < 2^34, but
        // only bits 29 .. 29 + v - 1 are wanted, so 32 bits suffice: for v = 3
        // they are bits 29..31 of X mod 2^32; for v = 4, bits 28..31 of
        // X / 2 = 8 z + floor(3 (q0 + 1) / 2) mod 2^32 (2^v z is even).  The
        // only wrap past 2^32 comes from a lazy z >= p, whose strip bits are 0
        // either way.  No wide multiply: the FMA-heavy pipe, which the step's
        // products keep busy, is spared.
        static_assert(v == 3 || v == 4, "thread-per-stream strips are 3 or 4 bits");
        constexpr int top = v == 4 ? 28 : 29;
        const uint32_t q0 = z >> (29 - v);
        const uint32_t x = v == 4 ? 8u * z + ((3u * q0 + 3u) >> 1) : 8u * z + 3u * q0 + 3u;
        uint32_t y;
        if constexpr (pos <= top) y = x >> (top - pos);
        else y = x << (pos - top);
        constexpr uint32_t mask = pos + v <= 32 ? ((1u << v) - 1u) << pos : 0xFFFFFFFFu << pos;
        return (y & mask) | w;
    }
}

// ----------------------------------------------------------------- jumps
// M = [[k, -q], [1, 0]] acting on (z^(n), z^(n-1)); tab[b] = M^(2^b) mod p.
template <int GEN>
__global__ void gm_table_kernel(uint64_t *tab)
{
    using P = GmT<GEN>;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t m0 = P::k % P::p, m1 = P::p - P::q % P::p, m2 = 1, m3 = 0;
#pragma unroll 1
    for (int b = 0; b < kJumpBits; ++b) {
        tab[4 * b] = m0; tab[4 * b + 1] = m1; tab[4 * b + 2] = m2; tab[4 * b + 3] = m3;
        uint64_t n0 = addmod_p<P::kind>(mulmod_p<P::kind>(m0, m0), mulmod_p<P::kind>(m1, m2));
        uint64_t n1 = addmod_p<P::kind>(mulmod_p<P::kind>(m0, m1), mulmod_p<P::kind>(m1, m3));
        uint64_t n2 = addmod_p<P::kind>(mulmod_p<P::kind>(m2, m0), mulmod_p<P::kind>(m3, m2));
        uint64_t n3 = addmod_p<P::kind>(mulmod_p<P::kind>(m2, m1), mulmod_p<P::kind>(m3, m3));
        m0 = n0; m1 = n1; m2 = n2; m3 = n3;
    }
}

template <int GEN>
__device__ __forceinline__ void gm_apply(const uint64_t *M, uint64_t &zc, uint64_t &zp)
{
    using P = GmT<GEN>;
    uint64_t c = addmod_p<P::kind>(mulmod_p<P::kind>(M[0], zc), mulmod_p<P::kind>(M[1], zp));
    uint64_t q = addmod_p<P::kind>(mulmod_p<P::kind>(M[2], zc), mulmod_p<P::kind>(M[3], zp));
    zc = c; zp = q;
}

// Jump by the 128-bit exponent (hi, lo), and by a third word w2 (bits 128..191).
template <int GEN>
__device__ __forceinline__ void gm_jump128(const uint64_t *tab, uint64_t lo, uint64_t hi, uint64_t &zc, uint64_t &zp,
                                           uint64_t w2 = 0)
{
#pragma unroll 1
    for (int b = 0; b < 64; ++b)
        if ((lo >> b) & 1u) gm_apply<GEN>(tab + 4 * b, zc, zp);
#pragma unroll 1
    for (int b = 0; b < 64; ++b)
        if ((hi >> b) & 1u) gm_apply<GEN>(tab + 4 * (64 + b), zc, zp);
#pragma unroll 1
    for (int b = 0; w2 && b < 64; ++b)
        if ((w2 >> b) & 1u) gm_apply<GEN>(tab + 4 * (128 + b), zc, zp);
}

// R = A B (2x2, row-major, mod p).
template <int GEN>
__device__ __forceinline__ void gm_mat_mul(uint64_t R[4], const uint64_t A[4], const uint64_t *B)
{
    using P = GmT<GEN>;
    const uint64_t r0 = addmod_p<P::kind>(mulmod_p<P::kind>(A[0], B[0]), mulmod_p<P::kind>(A[1], B[2]));
    const uint64_t r1 = addmod_p<P::kind>(mulmod_p<P::kind>(A[0], B[1]), mulmod_p<P::kind>(A[1], B[3]));
    const uint64_t r2 = addmod_p<P::kind>(mulmod_p<P::kind>(A[2], B[0]), mulmod_p<P::kind>(A[3], B[2]));
    const uint64_t r3 = addmod_p<P::kind>(mulmod_p<P::kind>(A[2], B[1]), mulmod_p<P::kind>(A[3], B[3]));
    R[0] = r0; R[1] = r1; R[2] = r2; R[3] = r3;
}

// M^e mod p for the exponent (hi, lo) from the table (M^(2^b) for each set
// bit; powers of one matrix commute, so the order of the products is free).
template <int GEN>
__device__ __forceinline__ void gm_matpow128(const uint64_t *tab, uint64_t lo, uint64_t hi, uint64_t R[4])
{
    R[0] = 1; R[1] = 0; R[2] = 0; R[3] = 1;
#pragma unroll 1
    for (int b = 0; b < 64; ++b)
        if ((lo >> b) & 1u) gm_mat_mul<GEN>(R, R, tab + 4 * b);
#pragma unroll 1
    for (int b = 0; hi && b < 64; ++b)
        if ((hi >> b) & 1u) gm_mat_mul<GEN>(R, R, tab + 4 * (64 + b));
}

__device__ __forceinline__ void mul64x64(uint64_t a, uint64_t b, uint64_t &lo, uint64_t &hi)
{
    lo = a * b;
    hi = __umul64hi(a, b);
}

// Base ensemble: lane i < s gets the base pair advanced by i * D (D: 128 bits).
template <int GEN>
__global__ void gm_seed_kernel(const uint64_t *tab, uint64_t *base, uint64_t seed, uint64_t dlo, uint64_t dhi)
{
    using P = GmT<GEN>;
    int i = threadIdx.x;
    if (blockIdx.x != 0 || i >= P::s) return;
    uint64_t a = 1, b = 1;
    if (seed != PRAND_SEED_DEFAULT) {
        uint64_t sm = seed;
        do { a = splitmix64_next(sm) % P::p; b = splitmix64_next(sm) % P::p; } while (!(a | b));
    }
    uint64_t zp = a, zc = b;  // (z^(0), z^(1))
    // e = i * D as 128 bits (s D fits inside the period p^2 - 1 < 2^122)
    uint64_t elo, ehi;
    mul64x64(dlo, (uint64_t)i, elo, ehi);
    ehi += dhi * (uint64_t)i;
    gm_jump128<GEN>(tab, elo, ehi, zc, zp);
    base[i] = zp << P::t;          // x^(n-1)
    base[P::s + i] = zc << P::t;   // x^(n)
}

// Stream j of the handle = base advanced by (first + j) * L, L of 128 bits (the
// exponent, of up to 192 bits, is exact).  One thread per point of a stream.
template <int GEN>
__global__ void gm_init_kernel(const uint64_t *tab, const uint64_t *base, uint64_t *state, uint64_t first, uint64_t n,
                               uint64_t llo, uint64_t lhi)
{
    using P = GmT<GEN>;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t g = tid / P::s;
    const int i = (int)(tid % P::s);
    if (g >= n) return;
    uint64_t zp = base[i] >> P::t, zc = base[P::s + i] >> P::t;
    const uint64_t k = first + g;
    uint64_t e0, c0, e1, c1;
    mul64x64(k, llo, e0, c0);
    mul64x64(k, lhi, e1, c1);
    e1 += c0;
    const uint64_t e2 = c1 + (e1 < c0 ? 1u : 0u);
    gm_jump128<GEN>(tab, e0, e1, zc, zp, e2);
    state[g * P::s + i] = zp << P::t;
    state[(n + g) * P::s + i] = zc << P::t;
}

template <int GEN>
__global__ void gm_skip_kernel(const uint64_t *tab, uint64_t *state, uint64_t n, U256 off)
{
    using P = GmT<GEN>;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t g = tid / P::s;
    const int i = (int)(tid % P::s);
    if (g >= n) return;
    uint64_t zp = state[g * P::s + i] >> P::t, zc = state[(n + g) * P::s + i] >> P::t;
#pragma unroll 1
    for (int b = 0; b < kJumpBits; ++b)
        if (u256_bit(off, b)) gm_apply<GEN>(tab + 4 * b, zc, zp);
    state[g * P::s + i] = zp << P::t;
    state[(n + g) * P::s + i] = zc << P::t;
}

// ----------------------------------------------------------------- generation
// Lane per point (v = 1): one step of the lane's point and the warp's output
// word (lane i <-> bit i), which every lane ends with.
template <int GEN>
__device__ __forceinline__ uint32_t gm_next_word(GmZ<GEN> &zc, GmZ<GEN> &zp)
{
    static_assert(GmT<GEN>::lanes == 32 && GmT<GEN>::s == 32, "lane-per-point ensembles have 32 points");
    if constexpr (GEN == PRAND_GM61) {  // (zc, zp) hold the rotated values u
        return __ballot_sync(kFull, gm61_step(zc, zp));
    } else {
        const GmZ<GEN> zn = gm_step<GEN>(zc, zp);
        zp = zc;
        zc = zn;
        return __ballot_sync(kFull, gm_strip1<GEN>(zn));
    }
}

// One warp generates `len` outputs of one section into o: rounds of 128 words;
// lane li keeps words 4 li .. 4 li + 3 of a round and stores them together, so
// the warp writes 512 contiguous bytes per round.  The lane that owns words
// 4c..4c+3 parks them in its own 16-byte shared-memory slot (a predicated store
// instead of four register selects).  Full rounds run without bounds checks;
// the last, partial round steps exactly the remaining count, so every point
// takes exactly `len` steps.  VEC: o is 16-byte aligned (32 for doubles) at
// every round start, so full rounds leave as one vector store per lane; the two
// store forms are separate instantiations (a run-time branch between two
// stores of the same values to the same addresses may be folded into the wider
// one).  zc, zp: the lane's point, canonical on entry and on return.
// Words per unrolled pass of a round's loop: four, except for GM61's f32 fill,
// which measured 1 % faster at two (its u32 fill 1 % slower).
template <int GEN, typename OutT>
__host__ __device__ constexpr int gm_round_unroll() { return GEN == PRAND_GM61 && std::is_same<OutT, float>::value ? 2 : 4; }

template <int GEN, typename OutT, bool VEC>
__device__ __forceinline__ void gm_generate_section(uint64_t &zc64, uint64_t &zp64, int li, OutT *o, uint64_t len,
                                                    uint32_t *myslot)
{
    constexpr int G = 32;
    constexpr int U = gm_round_unroll<GEN, OutT>();
    GmZ<GEN> zc, zp;
    if constexpr (GEN == PRAND_GM61) { zc = gm61_enter(zc64); zp = gm61_enter(zp64); }
    else { zc = (GmZ<GEN>)zc64; zp = (GmZ<GEN>)zp64; }
    const uint64_t full = len / (4 * G);
    for (uint64_t r = 0; r < full; ++r) {
#pragma unroll U
        for (int c = 0; c < G; ++c) {
            const uint32_t a = gm_next_word<GEN>(zc, zp);
            const uint32_t b = gm_next_word<GEN>(zc, zp);
            const uint32_t d = gm_next_word<GEN>(zc, zp);
            const uint32_t e = gm_next_word<GEN>(zc, zp);
            if (c == li) *reinterpret_cast<uint4 *>(myslot) = make_uint4(a, b, d, e);
        }
        const uint4 wv = *reinterpret_cast<const uint4 *>(myslot);
        OutT *q = o + r * 4 * G + 4 * li;
        if (VEC) {
            store4<OutT>(q, Cvt<OutT>::f(wv.x), Cvt<OutT>::f(wv.y), Cvt<OutT>::f(wv.z), Cvt<OutT>::f(wv.w));
        } else {
            q[0] = Cvt<OutT>::f(wv.x); q[1] = Cvt<OutT>::f(wv.y); q[2] = Cvt<OutT>::f(wv.z); q[3] = Cvt<OutT>::f(wv.w);
        }
    }
    const uint32_t rem = (uint32_t)(len - full * 4 * G);  // < 4 G
    if (rem) {
        uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
        for (uint32_t k = 0; k < rem; ++k) {
            const uint32_t w = gm_next_word<GEN>(zc, zp);
            if ((k >> 2) == (uint32_t)li) {
                const uint32_t u = k & 3u;
                w0 = u == 0 ? w : w0; w1 = u == 1 ? w : w1; w2 = u == 2 ? w : w2; w3 = u == 3 ? w : w3;
            }
        }
        OutT *q = o + full * 4 * G + 4 * li;
        const uint32_t pos = 4 * li;
        if (pos < rem) q[0] = Cvt<OutT>::f(w0);
        if (pos + 1 < rem) q[1] = Cvt<OutT>::f(w1);
        if (pos + 2 < rem) q[2] = Cvt<OutT>::f(w2);
        if (pos + 3 < rem) q[3] = Cvt<OutT>::f(w3);
    }
    if constexpr (GEN == PRAND_GM61) { zc64 = gm61_leave(zc); zp64 = gm61_leave(zp); }
    else { zc64 = gm_canon<GEN>(zc); zp64 = gm_canon<GEN>(zp); }
}

// One warp = one section of one stream.  The warp of the last section holds
// the stream's next state and writes it to state_out (a separate buffer when a
// stream is split into several sections, so no warp reads a state another
// warp has already replaced).
//
// Residency: GM61, GM29 and GM31 keep their pipes busiest with eight 256-thread
// blocks per SM (32 registers; ptxas moves a few loop-invariant words to the
// stack); GM19 and GQ58.1 run best at six (40 registers).
template <int GEN>
constexpr int gm_blocks_per_sm() { return GEN == PRAND_GM61 || GEN == PRAND_GM29 || GEN == PRAND_GM31 ? 8 : 6; }

template <int GEN, typename OutT, bool VEC>
__global__ void __launch_bounds__(256, gm_blocks_per_sm<GEN>()) gm_gen_kernel(const uint64_t *__restrict__ tab, const uint64_t *state_in,
                                                     uint64_t *state_out, uint64_t nstreams, uint64_t stride,
                                                     uint64_t nper, uint32_t nsec, uint64_t seclen,
                                                     OutT *__restrict__ out)
{
    using P = GmT<GEN>;
    __shared__ __align__(16) uint32_t slots[256 * 4];
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int li = threadIdx.x % 32;
    if (gid >= nstreams * nsec) return;  // gid is uniform within a warp
    const uint64_t j = gid % nstreams;
    const uint64_t start = (gid / nstreams) * seclen;
    if (start >= nper) return;
    const uint64_t len = min(seclen, nper - start);
    uint64_t zp = state_in[j * P::s + li] >> P::t;
    uint64_t zc = state_in[(stride + j) * P::s + li] >> P::t;
    if (start) gm_jump128<GEN>(tab, start, 0, zc, zp);
    gm_generate_section<GEN, OutT, VEC>(zc, zp, li, out + j * nper + start, len, slots + 4 * threadIdx.x);
    if (start + len == nper) {
        state_out[j * P::s + li] = zp << P::t;
        state_out[(stride + j) * P::s + li] = zc << P::t;
    }
}

// Thread per stream (v = 3, 4): every point of the thread's stream takes one
// step per output word; point I's strip goes to bit v I.
template <int GEN, int I>
__device__ __forceinline__ uint32_t gmt_point(GmZ<GEN> &zc, GmZ<GEN> &zp, uint32_t w)
{
    const GmZ<GEN> zn = gm_step<GEN>(zc, zp);
    zp = zc;
    zc = zn;
    return gm_strip_insert<GEN, I>(zn, w);
}
template <int GEN, int... I>
__device__ __forceinline__ uint32_t gmt_word(GmZ<GEN> *zc, GmZ<GEN> *zp, std::integer_sequence<int, I...>)
{
    uint32_t w = 0;
    ((w = gmt_point<GEN, I>(zc[I], zp[I], w)), ...);
    return w;
}
template <int GEN>
__device__ __forceinline__ uint32_t gmt_next_word(GmZ<GEN> *zc, GmZ<GEN> *zp)
{
    return gmt_word<GEN>(zc, zp, std::make_integer_sequence<int, GmT<GEN>::s>{});
}

// Load one stream's points (x >> t) from xp, xc and advance them by the
// exponent (hi, lo) with one matrix M^e applied to every point; canonical
// residues in and out.
template <int GEN>
__device__ __forceinline__ void gmt_load(const uint64_t *tab, const uint64_t *xp, const uint64_t *xc, uint64_t lo,
                                         uint64_t hi, GmZ<GEN> *zc, GmZ<GEN> *zp)
{
    using P = GmT<GEN>;
    uint64_t c[P::s], q[P::s];
#pragma unroll
    for (int i = 0; i < P::s; ++i) { q[i] = xp[i] >> P::t; c[i] = xc[i] >> P::t; }
    if (lo | hi) {
        uint64_t M[4];
        gm_matpow128<GEN>(tab, lo, hi, M);
#pragma unroll
        for (int i = 0; i < P::s; ++i) gm_apply<GEN>(M, c[i], q[i]);
    }
#pragma unroll
    for (int i = 0; i < P::s; ++i) { zc[i] = (GmZ<GEN>)c[i]; zp[i] = (GmZ<GEN>)q[i]; }
}

template <int GEN>
__device__ __forceinline__ void gmt_store(const GmZ<GEN> *zc, const GmZ<GEN> *zp, uint64_t *xp, uint64_t *xc)
{
    using P = GmT<GEN>;
#pragma unroll
    for (int i = 0; i < P::s; ++i) {
        xp[i] = gm_canon<GEN>(zp[i]) << P::t;
        xc[i] = gm_canon<GEN>(zc[i]) << P::t;
    }
}

// One thread = one section of one stream (sections reached by M^start).
// ROWS: every row start is 16-byte aligned, so rows leave through the staged
// 128-byte row stores (every lane of a warp takes part); else one store per
// output.  The thread of the last section writes the next state to state_out.
template <int GEN, typename OutT, bool ROWS>
__global__ void __launch_bounds__(256) gmt_gen_kernel(const uint64_t *__restrict__ tab, const uint64_t *state_in,
                                                      uint64_t *state_out, uint64_t nstreams, uint64_t stride,
                                                      uint64_t nper, uint32_t nsec, uint64_t seclen,
                                                      OutT *__restrict__ out)
{
    using P = GmT<GEN>;
    using Z = GmZ<GEN>;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = tid < nstreams * nsec;
    const uint64_t j = live ? tid % nstreams : 0;
    const uint64_t start = live ? (tid / nstreams) * seclen : 0;
    const uint64_t len = (live && start < nper) ? min(seclen, nper - start) : 0;
    Z zc[P::s], zp[P::s];
    if (len) {
        gmt_load<GEN>(tab, state_in + j * P::s, state_in + (stride + j) * P::s, start, 0, zc, zp);
    } else {
#pragma unroll
        for (int i = 0; i < P::s; ++i) { zc[i] = 0; zp[i] = 0; }
        if (!ROWS) return;
    }
    OutT *o = out + j * nper + start;
    if constexpr (ROWS) {
        __shared__ __align__(16) unsigned char tiles[256 / 32][kTileBytes];
        fill_rows<OutT, 128, true>([&]() { return gmt_next_word<GEN>(zc, zp); },
                                   [](uint32_t u) { return Cvt<OutT>::f(u); }, o, len, tiles[threadIdx.x >> 5],
                                   threadIdx.x & 31);
    } else {
        for (uint64_t i = 0; i < len; ++i) o[i] = Cvt<OutT>::f(gmt_next_word<GEN>(zc, zp));
    }
    if (len && start + len == nper) gmt_store<GEN>(zc, zp, state_out + j * P::s, state_out + (stride + j) * P::s);
}

// ----------------------------------------------------------------- host side
template <int GEN>
inline prand_status_t gm_build_table_t(uint64_t *tab, cudaStream_t st)
{
    gm_table_kernel<GEN><<<1, 32, 0, st>>>(tab);
    return launch_check();
}

inline unsigned gm_grid_for(uint64_t n, unsigned block) { return (unsigned)((n + block - 1) / block); }

template <int GEN>
struct GmHost {
    static prand_status_t seed(const uint64_t *tab, uint64_t *base, uint64_t seed, const Variant &V, cudaStream_t st)
    {
        gm_seed_kernel<GEN><<<1, 32, 0, st>>>(tab, base, seed, V.D[0], V.D[1]);
        return launch_check();
    }
    static prand_status_t init(const uint64_t *tab, const uint64_t *base, uint64_t *state, uint64_t first, uint64_t n,
                               const Variant &V, cudaStream_t st)
    {
        const unsigned B = 128;
        gm_init_kernel<GEN><<<gm_grid_for(n * GmT<GEN>::s, B), B, 0, st>>>(tab, base, state, first, n, V.L[0], V.L[1]);
        return launch_check();
    }
    static prand_status_t skip(const uint64_t *tab, uint64_t *state, uint64_t n, const U256 &off, cudaStream_t st)
    {
        const unsigned B = 128;
        gm_skip_kernel<GEN><<<gm_grid_for(n * GmT<GEN>::s, B), B, 0, st>>>(tab, state, n, off);
        return launch_check();
    }
    // Sections per stream: whole waves of the kernel's resident warps (lane
    // per point) or threads (thread per stream), cap; sections start on
    // multiples of 128 outputs (a warp's round) or 32 outputs (a 128-byte row).
    static void pick(uint64_t nstreams, uint64_t nper, uint64_t cap, uint32_t *nsec, uint64_t *seclen)
    {
        constexpr uint64_t A = GmT<GEN>::lanes == 32 ? 128 : 32;
        const uint32_t s = pick_nsec(nstreams, cap, GmT<GEN>::lanes == 32 ? nper / 512 : nper / 256, nper);
        uint64_t len = (nper + s - 1) / s;
        len = (len + A - 1) / A * A;
        if (len == 0) len = A;
        *seclen = len;
        *nsec = (uint32_t)((nper + len - 1) / len);
        if (*nsec == 0) *nsec = 1;
    }
    template <typename OutT>
    static prand_status_t gen(const uint64_t *tab, uint64_t *state, uint64_t *spare, StreamRange &R, OutT *out,
                              uint64_t nper, cudaStream_t st)
    {
        using P = GmT<GEN>;
        const unsigned B = 256;
        const uint64_t off = R.j0 * P::s;
        const uint64_t *sin = state + off;
        if constexpr (P::lanes == 32) {
            if (R.nsec == 0) pick(R.count, nper, resident_threads<GEN>(gm_gen_kernel<GEN, OutT, true>) / 32, &R.nsec, &R.seclen);
            const uint32_t nsec = R.nsec;
            const uint64_t seclen = R.seclen, nstreams = R.count;
            uint64_t *sout = (nsec > 1 ? spare : state) + off;
            // section starts are multiples of 128, so rows start 16-byte aligned
            // when the output is aligned and n_per_stream is a multiple of 4
            const bool vec = ((uintptr_t)out % (sizeof(OutT) == 8 ? 32 : 16)) == 0 && nper % 4 == 0;
            const unsigned grid = gm_grid_for(nstreams * nsec * 32, B);
            if (vec) gm_gen_kernel<GEN, OutT, true><<<grid, B, 0, st>>>(tab, sin, sout, nstreams, R.stride, nper, nsec, seclen, out);
            else gm_gen_kernel<GEN, OutT, false><<<grid, B, 0, st>>>(tab, sin, sout, nstreams, R.stride, nper, nsec, seclen, out);
        } else {
            if (R.nsec == 0) pick(R.count, nper, resident_threads<200 + GEN>(gmt_gen_kernel<GEN, OutT, true>), &R.nsec, &R.seclen);
            const uint32_t nsec = R.nsec;
            const uint64_t seclen = R.seclen, nstreams = R.count;
            uint64_t *sout = (nsec > 1 ? spare : state) + off;
            constexpr uint64_t E = RowFill<OutT>::E;
            const bool rows = ((uintptr_t)out % 16) == 0 && nper % E == 0 && seclen % E == 0;
            const unsigned grid = gm_grid_for(nstreams * nsec, B);
            if (rows) gmt_gen_kernel<GEN, OutT, true><<<grid, B, 0, st>>>(tab, sin, sout, nstreams, R.stride, nper, nsec, seclen, out);
            else gmt_gen_kernel<GEN, OutT, false><<<grid, B, 0, st>>>(tab, sin, sout, nstreams, R.stride, nper, nsec, seclen, out);
        }
        return launch_check();
    }
};


// Per-generator entry points, instantiated one translation unit per generator.
#define PRAND_GM_INSTANTIATE(GEN, NAME)                                                                          \
    prand_status_t NAME##_table(uint64_t *tab, cudaStream_t st) { return gm_build_table_t<GEN>(tab, st); }      \
    prand_status_t NAME##_seed(const uint64_t *tab, uint64_t *base, uint64_t seed, const Variant &V,           \
                               cudaStream_t st)                                                               \
    {                                                                                                         \
        return GmHost<GEN>::seed(tab, base, seed, V, st);                                                     \
    }                                                                                                         \
    prand_status_t NAME##_init(const uint64_t *tab, const uint64_t *base, uint64_t *state, uint64_t first,     \
                               uint64_t n, const Variant &V, cudaStream_t st)                                 \
    {                                                                                                         \
        return GmHost<GEN>::init(tab, base, state, first, n, V, st);                                          \
    }                                                                                                         \
    prand_status_t NAME##_skip(const uint64_t *tab, uint64_t *state, uint64_t n, const U256 &off,             \
                               cudaStream_t st)                                                               \
    {                                                                                                         \
        return GmHost<GEN>::skip(tab, state, n, off, st);                                                     \
    }                                                                                                         \
    prand_status_t NAME##_gen(const uint64_t *tab, uint64_t *state, uint64_t *spare, StreamRange &R,          \
                              void *out, int dtype, uint64_t nper, cudaStream_t st)                            \
    {                                                                                                         \
        if (dtype == PRAND_DTYPE_U32)                                                                         \
            return GmHost<GEN>::template gen<uint32_t>(tab, state, spare, R, (uint32_t *)out, nper, st); \
        if (dtype == PRAND_DTYPE_F32)                                                                         \
            return GmHost<GEN>::template gen<float>(tab, state, spare, R, (float *)out, nper, st);  \
        return GmHost<GEN>::template gen<double>(tab, state, spare, R, (double *)out, nper, st);    \
    }

}  // namespace prand
