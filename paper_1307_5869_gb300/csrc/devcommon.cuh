// Device helpers shared by the generation and jump kernels: exact modular
// arithmetic for the moduli of Sec. 5.1-5.2, SplitMix64 seed expansion, the
// float epilogue, and vectorised output emission.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "prand_internal.h"

namespace prand {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------- SplitMix64
// Seed expansion (Steele, Lea & Flood 2014); the same published definition on
// both sides of any comparison, used only to turn a 64-bit seed into states.
__host__ __device__ inline uint64_t splitmix64_next(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- mod m1, m2
// a * b mod m for m = 2^32 - c (c = 209 or 22853), a, b < 2^32: fold the high
// word twice with 2^32 = c (mod m).
template <uint32_t C>
__device__ __forceinline__ uint32_t mulmod_2p32_minus(uint32_t a, uint32_t b)
{
    constexpr uint64_t m = (1ull << 32) - C;
    uint64_t p = (uint64_t)a * b;
    uint64_t t = (p & 0xFFFFFFFFull) + (uint64_t)C * (p >> 32);   // < 2^32 (1 + C)
    t = (t & 0xFFFFFFFFull) + (uint64_t)C * (t >> 32);            // < 2^32 + C (C+1)
    if (t >= m) t -= m;
    return (uint32_t)t;
}

__device__ __forceinline__ uint32_t addmod_u32(uint32_t a, uint32_t b, uint32_t m)
{
    uint64_t s = (uint64_t)a + b;
    return (uint32_t)(s >= m ? s - m : s);
}

// ---------------------------------------------------------------- mod p (GM/GQ)
// Full products of residues modulo the five primes of Table 2.
template <int KIND>
__device__ __forceinline__ uint64_t reduce_prod(uint64_t lo, uint64_t hi);

// p = 2^19 - 1: product < 2^38 (hi = 0)
template <>
__device__ __forceinline__ uint64_t reduce_prod<P19>(uint64_t lo, uint64_t)
{
    constexpr uint64_t p = (1ull << 19) - 1;
    uint64_t r = (lo & p) + (lo >> 19);   // < 2^20
    r = (r & p) + (r >> 19);              // <= p + 1
    return r >= p ? r - p : r;
}
// p = 2^29 - 3: product < 2^58 (hi = 0); 2^29 = 3 (mod p)
template <>
__device__ __forceinline__ uint64_t reduce_prod<P29>(uint64_t lo, uint64_t)
{
    constexpr uint64_t p = (1ull << 29) - 3, m = (1ull << 29) - 1;
    uint64_t r = (lo & m) + 3 * (lo >> 29);   // < 2^29 + 3 * 2^29
    r = (r & m) + 3 * (r >> 29);              // < 2^29 + 12
    return r >= p ? r - p : r;
}
// p = 2^31 - 1: product < 2^62 (hi = 0)
template <>
__device__ __forceinline__ uint64_t reduce_prod<P31>(uint64_t lo, uint64_t)
{
    constexpr uint64_t p = (1ull << 31) - 1;
    uint64_t r = (lo & p) + (lo >> 31);   // < 2^32
    r = (r & p) + (r >> 31);
    return r >= p ? r - p : r;
}
// p = 2^51 - 129: product < 2^102; 2^51 = 129 (mod p)
template <>
__device__ __forceinline__ uint64_t reduce_prod<P51>(uint64_t lo, uint64_t hi)
{
    constexpr uint64_t p = (1ull << 51) - 129, m = (1ull << 51) - 1;
    uint64_t h = (hi << 13) | (lo >> 51);         // < 2^51
    uint64_t r = (lo & m) + 129 * h;              // < 2^51 + 2^59
    r = (r & m) + 129 * (r >> 51);                // < 2^51 + 2^17
    return r >= p ? r - p : r;
}
// p = 2^61 - 1: product < 2^122
template <>
__device__ __forceinline__ uint64_t reduce_prod<P61>(uint64_t lo, uint64_t hi)
{
    constexpr uint64_t p = (1ull << 61) - 1;
    uint64_t r = (lo & p) + ((hi << 3) | (lo >> 61));   // < 2^62
    r = (r & p) + (r >> 61);
    return r >= p ? r - p : r;
}

template <int KIND>
__device__ __forceinline__ uint64_t mulmod_p(uint64_t a, uint64_t b)
{
    if (KIND == P51 || KIND == P61) return reduce_prod<KIND>(a * b, __umul64hi(a, b));
    return reduce_prod<KIND>(a * b, 0);
}

template <int KIND>
__device__ __forceinline__ uint64_t prime_of()
{
    return KIND == P19 ? (1ull << 19) - 1 : KIND == P29 ? (1ull << 29) - 3 : KIND == P31 ? (1ull << 31) - 1
         : KIND == P51 ? (1ull << 51) - 129 : (1ull << 61) - 1;
}

template <int KIND>
__device__ __forceinline__ uint64_t addmod_p(uint64_t a, uint64_t b)
{
    uint64_t s = a + b;   // both < p < 2^62
    return s >= prime_of<KIND>() ? s - prime_of<KIND>() : s;
}

// ---------------------------------------------------------------- floats
// f32 = (u >> 8) * 2^-24, formed as (u & 0xFFFFFF00) * 2^-32: the masked word
// has at most 24 significant bits, so it converts exactly (in any rounding
// mode), and the scale is a power of two whose product stays normal (the
// smallest nonzero value is 2^-24).  The mask folds into the logic operation
// that forms u in the cheapest generators (LFSR113's XOR of its components),
// so no shift is spent on either integer pipe.
__device__ __forceinline__ float u32_to_f32(uint32_t u) { return __uint2float_rz(u & 0xFFFFFF00u) * 0x1p-32f; }

// f64 = u * 2^-32, assembled from the bits (exact) to stay off the FP64 pipe.
__device__ __forceinline__ double u32_to_f64(uint32_t u)
{
    if (u == 0) return 0.0;
    int lz = __clz(u);                         // MSB at bit 31 - lz
    uint32_t m = (u << lz) << 1;               // fraction bits, MSB dropped
    uint32_t hi = ((uint32_t)(1022 - lz) << 20) | (m >> 12);
    uint32_t lo = m << 20;
    return __hiloint2double((int)hi, (int)lo);
}

// MRG32K3A f64 = z * RN(1 / (m1 + 1)), one round-to-nearest multiply, done in
// integer arithmetic so it stays off the FP64 pipe.  The constant is
// M 2^-84 with M = 0x1000000D00000B (53 bits, high word 2^20), so the exact
// product is P 2^-84 with P = z 2^52 + z Ml (Ml = M mod 2^32, one wide
// multiply).  With top = P >> 32 of bit length L, the double keeps the 53 bits
// P >> s, s = L - 21, rounded to nearest even on the s dropped bits, and its
// bits are ((s + 990) << 52) + mantissa (a round-up to 2^53 carries into the
// exponent by itself).  z = 0 gives 0.
__device__ __forceinline__ double mrg_to_f64(uint32_t z)
{
    const uint64_t zm = (uint64_t)z * 0x0D00000Bu;               // z Ml < 2^60
    const uint32_t w0 = (uint32_t)zm;                             // P mod 2^32
    const uint64_t top = ((uint64_t)z << 20) + (zm >> 32);        // P >> 32 < 2^53
    const uint32_t th = (uint32_t)(top >> 32), tl = (uint32_t)top;
    const int L = th ? 64 - __clz(th) : 32 - __clz(tl);           // 21..53 for z >= 1
    const int sh = L - 21;                                        // bits dropped, 0..32
    uint32_t mlo, mhi;
    asm("shf.r.clamp.b32 %0, %2, %3, %4;\n\t"
        "shf.r.clamp.b32 %1, %3, %5, %4;"
        : "=r"(mlo), "=r"(mhi) : "r"(w0), "r"(tl), "r"(sh), "r"(th));
    // the dropped bits, left-aligned (0 when nothing is dropped); round up above
    // one half, or at one half when the kept part is odd
    const uint32_t rem = sh ? w0 << (32 - sh) : 0u;
    const uint32_t up = rem > 0x80000000u - (mlo & 1u) ? 1u : 0u;
    const uint64_t m = (((uint64_t)mhi << 32) | mlo) + up;
    const uint64_t bits = ((uint64_t)(sh + 990) << 52) + m;
    return z ? __longlong_as_double((long long)bits) : 0.0;
}

// ---------------------------------------------------------------- output
// Conversion of one 32-bit output to the requested element type.
template <typename OutT, bool MRG = false>
struct Cvt;
template <bool MRG>
struct Cvt<uint32_t, MRG> { __device__ __forceinline__ static uint32_t f(uint32_t u) { return u; } };
template <bool MRG>
struct Cvt<float, MRG> { __device__ __forceinline__ static float f(uint32_t u) { return u32_to_f32(u); } };
template <>
struct Cvt<double, false> { __device__ __forceinline__ static double f(uint32_t u) { return u32_to_f64(u); } };
template <>
struct Cvt<double, true> { __device__ __forceinline__ static double f(uint32_t u) { return mrg_to_f64(u); } };

// Store four consecutive elements at p (16-byte aligned for 4-byte types,
// 32-byte aligned for doubles when vec is true).
template <typename OutT>
__device__ __forceinline__ void store4(OutT *p, OutT a, OutT b, OutT c, OutT d);
template <>
__device__ __forceinline__ void store4<uint32_t>(uint32_t *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    *reinterpret_cast<uint4 *>(p) = make_uint4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store4<float>(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store4<double>(double *p, double a, double b, double c, double d)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}

// ---------------------------------------------------------------- row staging
// Thread-per-stream generators produce one row of outputs per lane; written
// directly, a warp store would scatter 32 small pieces over 32 rows.  Instead
// each lane stages ROWB bytes (128 or 256) of its row in a padded shared-memory
// tile (pitch ROWB + 16, so 16-byte accesses are bank-conflict free on both
// sides) and the warp writes the tile out as whole ROWB-byte row segments,
// 512 / ROWB rows per store.  Longer segments suit HBM better; shorter ones
// need half the shared memory.
template <typename OutT, int ROWB = 128>
struct RowFill {
    static constexpr int K = ROWB / (int)sizeof(OutT);  // outputs per row chunk
    static constexpr int E = 16 / (int)sizeof(OutT);    // outputs per 16-byte vector
    static constexpr int PITCH = ROWB + 16;             // tile bytes per row
    static constexpr int TILE = 32 * PITCH;             // tile bytes per warp
    static constexpr int PIECES = ROWB / 16;            // 16-byte pieces per row segment
    static constexpr int ROWS = 32 / PIECES;            // row segments per warp store
};
constexpr int kTileBytes = RowFill<uint32_t, 128>::TILE;  // per warp, 128-byte segments

// Emits `len` outputs of this lane's stream to dst (16-byte aligned rows), all
// 32 lanes of the warp taking part (lanes with len 0 only help store).
// next() returns the next 32-bit output; cvt converts it.  tile: the warp's
// RowFill<OutT, ROWB>::TILE bytes of shared memory.
// ROLL: keep the loop over a chunk's 16-byte pieces rolled (for generators
// whose next() is long, where unrolling a whole chunk would outgrow the
// instruction cache).
template <typename OutT, int ROWB = 128, bool ROLL = false, typename Next, typename Conv>
__device__ __forceinline__ void fill_rows(Next &&next, Conv &&cvt, OutT *dst, uint64_t len, unsigned char *tile, int lane)
{
    using RF = RowFill<OutT, ROWB>;
    constexpr int K = RF::K, E = RF::E, PITCH = RF::PITCH, PIECES = RF::PIECES, ROWS = RF::ROWS;
    uint64_t maxlen = len;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) maxlen = max(maxlen, (uint64_t)__shfl_xor_sync(kFull, (unsigned long long)maxlen, d));
    const uint64_t nch = (maxlen + K - 1) / K;
    unsigned char *myrow = tile + lane * PITCH;
    const int piece = lane % PIECES;
    for (uint64_t ch = 0; ch < nch; ++ch) {
        const uint32_t cnt = len > ch * K ? (uint32_t)min((uint64_t)K, len - ch * K) : 0u;
        const unsigned long long mydst = (unsigned long long)(dst + ch * K);
        if (__all_sync(kFull, cnt == (uint32_t)K)) {
            // every lane has a whole chunk: no per-output tests, and every row
            // segment of the tile is stored whole
#pragma unroll (ROLL ? 1 : PIECES)
            for (int v = 0; v < PIECES; ++v) {
                OutT vals[E];
#pragma unroll
                for (int e = 0; e < E; ++e) vals[e] = cvt(next());
                *reinterpret_cast<uint4 *>(myrow + 16 * v) = *reinterpret_cast<const uint4 *>(vals);
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < PIECES; ++i) {
                const int r = ROWS * i + lane / PIECES;
                OutT *rd = (OutT *)__shfl_sync(kFull, mydst, r);
                *reinterpret_cast<uint4 *>(rd + piece * E) = *reinterpret_cast<const uint4 *>(tile + r * PITCH + 16 * piece);
            }
            __syncwarp();
            continue;
        }
#pragma unroll
        for (int v = 0; v < PIECES; ++v) {
            if ((uint32_t)(v * E) < cnt) {
                OutT vals[E];
#pragma unroll
                for (int e = 0; e < E; ++e) vals[e] = (uint32_t)(v * E + e) < cnt ? cvt(next()) : OutT(0);
                *reinterpret_cast<uint4 *>(myrow + 16 * v) = *reinterpret_cast<const uint4 *>(vals);
            }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < PIECES; ++i) {
            const int r = ROWS * i + lane / PIECES;
            OutT *rd = (OutT *)__shfl_sync(kFull, mydst, r);
            const uint32_t rc = __shfl_sync(kFull, cnt, r);
            const int col = piece * E;
            const unsigned char *src = tile + r * PITCH + 16 * piece;
            if ((uint32_t)(col + E) <= rc) {
                *reinterpret_cast<uint4 *>(rd + col) = *reinterpret_cast<const uint4 *>(src);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((uint32_t)(col + e) < rc) rd[col + e] = reinterpret_cast<const OutT *>(src)[e];
            }
        }
        __syncwarp();
    }
}

// Resident threads of a kernel launched with BS-thread blocks on the current
// device, computed once per kernel and device (ID tells the kernels apart: the
// generator id for the per-handle fills, 100 and up for the others).
template <int ID, int BS = 256, typename K>
inline uint64_t resident_threads(K kernel)
{
    constexpr int kDevs = 64;
    static std::atomic<uint64_t> cache[kDevs];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < kDevs) {
        const uint64_t c = cache[dev].load(std::memory_order_relaxed);
        if (c) return c;
    }
    const int sms = device_sm_count();
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, BS, 0) != cudaSuccess || bps < 1) bps = 1;
    const uint64_t c = (uint64_t)sms * bps * BS;
    if (dev >= 0 && dev < kDevs) cache[dev].store(c, std::memory_order_relaxed);
    return c;
}

// Big offsets.
__device__ __forceinline__ int u256_bit(const U256 &e, int b) { return (int)((e.w[b >> 6] >> (b & 63)) & 1u); }

}  // namespace prand
