// Device routines of MRG32K3A (Sec. 5.2) and LFSR113 (Sec. 5.3) shared by the
// per-handle kernels and the batched persistent kernel: one recurrence step,
// and one jump-table application (bit b of an offset).
#pragma once
#include "devcommon.cuh"

namespace prand {

// =========================================================== MRG32K3A
// Matrices of Sec. 5.2 with the negative entries taken mod m.
__device__ __forceinline__ void mrg_step_matrices(uint32_t A[9], uint32_t B[9])
{
    const uint32_t a0[9] = { 0u, 1403580u, kM1 - 810728u, 1u, 0u, 0u, 0u, 1u, 0u };
    const uint32_t b0[9] = { 527612u, 0u, kM2 - 1370589u, 1u, 0u, 0u, 0u, 1u, 0u };
    for (int i = 0; i < 9; ++i) { A[i] = a0[i]; B[i] = b0[i]; }
}

template <uint32_t C>
__device__ void mat3_sqr(uint32_t M[9])
{
    constexpr uint32_t m = (uint32_t)((1ull << 32) - C);
    uint32_t R[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            uint32_t s = 0;
            for (int k = 0; k < 3; ++k) s = addmod_u32(s, mulmod_2p32_minus<C>(M[3 * i + k], M[3 * k + j]), m);
            R[3 * i + j] = s;
        }
    for (int i = 0; i < 9; ++i) M[i] = R[i];
}

template <uint32_t C>
__device__ __forceinline__ void mat3_vec(const uint32_t *M, uint32_t v[3])
{
    constexpr uint32_t m = (uint32_t)((1ull << 32) - C);
    uint32_t r[3];
    for (int i = 0; i < 3; ++i) {
        uint32_t s = 0;
        for (int k = 0; k < 3; ++k) s = addmod_u32(s, mulmod_2p32_minus<C>(M[3 * i + k], v[k]), m);
        r[i] = s;
    }
    v[0] = r[0]; v[1] = r[1]; v[2] = r[2];
}

// Apply the jump of bit b of the table to (x, y).
__device__ __forceinline__ void mrg_apply_bit(const uint32_t *tab, int b, uint32_t x[3], uint32_t y[3])
{
    mat3_vec<209>(tab + 18 * b, x);
    mat3_vec<22853>(tab + 18 * b + 9, y);
}

// One MRG32K3A step (x_n = a x_{n-2} - b x_{n-3} mod m1, y_n = c y_{n-1} -
// d y_{n-3} mod m2, Sec. 5.2) on canonical residues, in 32-bit limbs:
// t = m - v (no borrow), S = A u + B t < 2^54 by two wide multiply-adds; with
// 2^32 = e (mod m) (e = 209 or 22853) S folds to lo + e hi (for m2 twice, the
// first fold's e hi by a wide multiply with lo added by a carry chain, the
// second high word being below 2^6); then r < 2^32 + 2^30 is made canonical as
// r + e [r >= m], the condition being the carry out of r + e.
// Returns z = x_n - y_n mod m1 in [1, m1].
__device__ __forceinline__ uint32_t mrg_next(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                             uint32_t &y0, uint32_t &y1, uint32_t &y2)
{
    uint32_t xn, yn;
    asm("{\n\t"
        ".reg .u32 t, lo, hi, p, r, c, q;\n\t"
        ".reg .u64 T, U;\n\t"
        "sub.u32 t, 4294967087, %2;\n\t"
        "mul.wide.u32 T, t, 810728;\n\t"
        "mad.wide.u32 U, %1, 1403580, T;\n\t"
        "mov.b64 {lo, hi}, U;\n\t"
        "mul.lo.u32 p, hi, 209;\n\t"
        "add.cc.u32 r, lo, p;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "add.cc.u32 q, r, 209;\n\t"
        "addc.u32 c, c, 0;\n\t"
        "mad.lo.u32 %0, c, 209, r;\n\t"
        "}"
        : "=r"(xn) : "r"(x1), "r"(x2));
    asm("{\n\t"
        ".reg .u32 t, lo, hi, s0, s1, p0, p1, p, r, c, q;\n\t"
        ".reg .u64 T, W, P;\n\t"
        "sub.u32 t, 4294944443, %2;\n\t"
        "mul.wide.u32 T, t, 1370589;\n\t"
        "mad.wide.u32 W, %1, 527612, T;\n\t"
        "mov.b64 {lo, hi}, W;\n\t"
        "mul.wide.u32 P, hi, 22853;\n\t"
        "mov.b64 {p0, p1}, P;\n\t"
        "add.cc.u32 s0, p0, lo;\n\t"
        "addc.u32 s1, p1, 0;\n\t"
        "mul.lo.u32 p, s1, 22853;\n\t"
        "add.cc.u32 r, s0, p;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "add.cc.u32 q, r, 22853;\n\t"
        "addc.u32 c, c, 0;\n\t"
        "mad.lo.u32 %0, c, 22853, r;\n\t"
        "}"
        : "=r"(yn) : "r"(y0), "r"(y2));
    x2 = x1; x1 = x0; x0 = xn;
    y2 = y1; y1 = y0; y0 = yn;
    return xn > yn ? xn - yn : xn - yn + kM1;
}


// =========================================================== LFSR113
// Component (p, q, s): (31,6,18), (29,2,2), (28,13,7), (25,3,13).  The word
// holds bits x_{ns}..x_{ns+31} of eq. (lfsrOutput); a step keeps the top p bits
// shifted by s and refills the rest through eq. (lfsrRel1).
template <int P, int Q, int S>
__host__ __device__ __forceinline__ uint32_t taus_step(uint32_t z)
{
    constexpr uint32_t mask = 0xFFFFFFFFu << (32 - P);
    return ((z & mask) << S) ^ (((z << Q) ^ z) >> (P - S));
}

__device__ __forceinline__ uint32_t lfsr_comp_step(int c, uint32_t z)
{
    switch (c) {
    case 0: return taus_step<31, 6, 18>(z);
    case 1: return taus_step<29, 2, 2>(z);
    case 2: return taus_step<28, 13, 7>(z);
    default: return taus_step<25, 3, 13>(z);
    }
}

__device__ __forceinline__ uint32_t gf2_apply(const uint32_t *col, uint32_t v)
{
    uint32_t r = 0;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) r ^= ((v >> i) & 1u) ? col[i] : 0u;
    return r;
}

// The lookups depend only on the bit b, so every lane of a warp reads the same
// 32 words: one broadcast per word, whatever the lanes' states.
__device__ __forceinline__ void lfsr_apply_bit(const uint32_t *tab, int b, uint32_t z[4])
{
    for (int c = 0; c < 4; ++c) z[c] = gf2_apply(tab + ((size_t)c * kJumpBits + b) * 32, z[c]);
}

// The same word step with one funnel shift: the masked part, (z & mask) << S,
// holds bits [32 - R, 32) and ((z << Q) ^ z) >> R bits [0, 32 - R) (R = P - S),
// so the new word is the low half of the 64-bit value (z >> (32 - P) : b) >> R,
// b = (z << Q) ^ z -- four operations instead of five.  The combined step is
// bound by the integer ALU pipe: z << Q is written as the multiply z 2^Q (the
// multiply pipe), and with HI, z >> (32 - P) as the high word of z 2^P
// (P <= 31), a multiply that holds the multiply pipe twice as long, so only
// two of the four components take it.
template <int P, int Q, int S, bool HI>
__device__ __forceinline__ uint32_t taus_step_funnel(uint32_t z)
{
    uint32_t lo, hi;
    if constexpr (HI) {
        asm("mul.lo.u32 %0, %2, %3;\n\t"
            "mul.hi.u32 %1, %2, %4;"
            : "=r"(lo), "=r"(hi) : "r"(z), "n"(1u << Q), "n"(1u << P));
    } else {
        asm("mul.lo.u32 %0, %1, %2;" : "=r"(lo) : "r"(z), "n"(1u << Q));
        hi = z >> (32 - P);
    }
    return __funnelshift_r(lo ^ z, hi, P - S);
}

__device__ __forceinline__ uint32_t lfsr_next(uint32_t &z0, uint32_t &z1, uint32_t &z2, uint32_t &z3)
{
    z0 = taus_step_funnel<31, 6, 18, true>(z0);
    z1 = taus_step_funnel<29, 2, 2, false>(z1);
    z2 = taus_step_funnel<28, 13, 7, true>(z2);
    z3 = taus_step_funnel<25, 3, 13, false>(z3);
    return z0 ^ z1 ^ z2 ^ z3;
}


}  // namespace prand
