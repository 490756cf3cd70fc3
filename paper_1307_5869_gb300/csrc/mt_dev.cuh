// Device routines of MT19937 (Matsumoto & Nishimura 1998; Sec. 5.4) shared by
// the per-handle kernels and the batched persistent kernel: the recurrence
// word, tempering, the fused twist-and-emit of one block, and the polynomial
// jump of eq. (g_v) applied by one warp.
#pragma once
#include "devcommon.cuh"

namespace prand {

__device__ __forceinline__ uint32_t mt_recur(uint32_t xt, uint32_t xt1, uint32_t xt397)
{
    uint32_t y = (xt & 0x80000000u) | (xt1 & 0x7FFFFFFFu);
    return xt397 ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
}

// Copy one 624-word state with a warp: all of a lane's 20 loads are issued
// before any of its stores, so the copy costs one memory latency rather than
// twenty.  Each lane moves its own words (src and dst may be the same buffer).
__device__ __forceinline__ void mt_copy_state_warp(const uint32_t *src, uint32_t *dst, int lane)
{
    constexpr int R = (kMtN + 31) / 32;  // 20
    uint32_t r[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = lane + 32 * k;
        r[k] = i < kMtN ? src[i] : 0u;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = lane + 32 * k;
        if (i < kMtN) dst[i] = r[k];
    }
}

__device__ __forceinline__ uint32_t mt_temper(uint32_t y)
{
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

// Twist of a whole block out of place (old block -> new block, both in shared
// memory) fused with the tempered output: every new word is tempered and
// stored straight from registers while it is written to the new block.  New
// word k reads old words k, k+1 (new word 0 for k = 623) and old word k + 397
// (k < 227) or new word k - 227 (k >= 227).  So the block is made in 20 chunks
// of 32 words in order.  The loop is unrolled completely so each chunk knows
// its case at compile time (only chunk 7 mixes the two partner sources and
// only chunk 19 is partly empty).  A word read from the new block was written
// at least seven chunks earlier, so a warp sync every fourth chunk orders
// every such read after its write.  Words k < emit are written to o[k]; FULL
// (emit == 624) drops that test.
template <typename OutT, bool FULL>
__device__ __forceinline__ void mt_twist_emit_chunks(const uint32_t *__restrict__ ob, uint32_t *__restrict__ nb,
                                                     int lane, OutT *o, uint32_t emit)
{
#pragma unroll
    for (int c = 0; c < 20; ++c) {
        const int k = 32 * c + lane;
        if (c < 19 || lane < kMtN - 32 * 19) {
            const uint32_t a = ob[k];
            const uint32_t b = (c < 19 || lane < kMtN - 32 * 19 - 1) ? ob[k + 1] : nb[0];
            const uint32_t p = c < 7 ? ob[k + 397] : c > 7 ? nb[k - 227] : (lane < 3 ? ob[k + 397] : nb[k - 227]);
            const uint32_t x = mt_recur(a, b, p);
            nb[k] = x;
            if (FULL || (uint32_t)k < emit) o[k] = Cvt<OutT>::f(mt_temper(x));
        }
        if ((c & 3) == 3) __syncwarp();
    }
}

template <typename OutT>
__device__ __forceinline__ void mt_twist_emit(const uint32_t *__restrict__ ob, uint32_t *__restrict__ nb, int lane,
                                              OutT *o, uint32_t emit)
{
    if (emit >= (uint32_t)kMtN) mt_twist_emit_chunks<OutT, true>(ob, nb, lane, o, emit);
    else mt_twist_emit_chunks<OutT, false>(ob, nb, lane, o, emit);
}

// Twist of one block out of place (no output): the 20-chunk in-order schedule
// of mt_twist_emit_chunks, kept as a compact loop (it runs inside the jump's
// unrolled sliding-window loop, where code size matters more than its cost).
__device__ __forceinline__ void mt_twist_block(const uint32_t *ob, uint32_t *nb, int lane)
{
#pragma unroll 4
    for (int c = 0; c < 20; ++c) {
        const int k = 32 * c + lane;
        if (k < kMtN) {
            const uint32_t b = k + 1 < kMtN ? ob[k + 1] : nb[0];
            const uint32_t p = k < 227 ? ob[k + 397] : nb[k - 227];
            nb[k] = mt_recur(ob[k], b, p);
        }
        if ((c & 3) == 3) __syncwarp();
    }
}

// dst := g(A) src for one stream, by one warp (eq. (g_v)).  With src in window
// form x_0..x_623, A^i src is the window x_i..x_{i+623}, so result word m is the
// XOR of x_{i+m} over the set coefficients i of g.  Lane l owns 20 consecutive
// result words m = mbase + j (mbase = 20 l, and 604 for lane 31, whose first 16
// words repeat lane 30's) and keeps the 20 sequence words x_{i+mbase..i+mbase+19}
// in registers as a window that slides by one word per coefficient: one
// shared-memory load per coefficient, and 20 register XORs per set coefficient
// (one three-input XOR when two neighbouring coefficients are both set).
// seq is a 1248-word ring holding two consecutive 624-word blocks (x at index
// i sits at seq[i mod 1248]); the block two ahead is twisted into the oldest
// slot once no lane will load from it again (loads at step i reach x_{i+19}
// .. x_{i+623}).  src may equal dst or seq.
__device__ inline void mt_apply_poly_warp(const uint32_t *__restrict__ poly, const uint32_t *src, uint32_t *dst,
                                          uint32_t *seq, int lane)
{
    constexpr int W = 20, RING = 2 * kMtN;
    const int mbase = lane < 31 ? W * lane : kMtN - W;
    uint32_t acc[W], win[W];
#pragma unroll
    for (int j = 0; j < W; ++j) acc[j] = 0;
    mt_copy_state_warp(src, seq, lane);
    __syncwarp();
    mt_twist_block(seq, seq + kMtN, lane);  // block 1 into slot 1
#pragma unroll
    for (int j = 0; j < W - 1; ++j) win[j] = seq[mbase + j];
    int next_block = 2;
    int p0 = mbase + W - 1;  // ring position of the word loaded at step i0
    for (int i0 = 0; i0 < kMtDeg; i0 += W) {
        if (next_block <= 32 && i0 >= kMtN * (next_block - 2) + 605) {
            __syncwarp();
            mt_twist_block(seq + ((next_block - 1) & 1) * kMtN, seq + (next_block & 1) * kMtN, lane);
            ++next_block;
        }
        const int w = i0 >> 5, sh = i0 & 31;
        const uint64_t two = (uint64_t)__ldg(poly + w) | ((uint64_t)(w + 1 < kMtPolyWords ? __ldg(poly + w + 1) : 0u) << 32);
        const uint32_t bits = (uint32_t)(two >> sh) & ((1u << W) - 1u);
#pragma unroll
        for (int u = 0; u < W; u += 2) {
            // step u: window slots (u + j) % W hold x_{i0+u+mbase+j}; the newest,
            // x_{i0+u+mbase+19}, goes into slot (u + 19) % W.  Step u + 1 needs
            // x_{i0+u+1+mbase+19} as its j = 19 word (nx); it replaces the oldest
            // word (slot u % W) only after both steps are applied.
            int pa = p0 + u, pb = p0 + u + 1;
            if (pa >= RING) pa -= RING;
            if (pb >= RING) pb -= RING;
            win[(u + W - 1) % W] = seq[pa];
            const uint32_t nx = seq[pb];
            const uint32_t pat = (bits >> u) & 3u;
            if (pat == 1u) {
#pragma unroll
                for (int j = 0; j < W; ++j) acc[j] ^= win[(u + j) % W];
            } else if (pat == 2u) {
#pragma unroll
                for (int j = 0; j < W; ++j) acc[j] ^= (j < W - 1 ? win[(u + 1 + j) % W] : nx);
            } else if (pat == 3u) {
#pragma unroll
                for (int j = 0; j < W; ++j) acc[j] ^= win[(u + j) % W] ^ (j < W - 1 ? win[(u + 1 + j) % W] : nx);
            }
            win[u % W] = nx;
        }
        p0 += W;
        if (p0 >= RING) p0 -= RING;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (lane < 31 || j >= W - 4) dst[mbase + j] = acc[j];
    __syncwarp();
}

}  // namespace prand
