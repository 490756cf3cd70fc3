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

// The same twist by a team of TEAM warps that make up the whole block (TEAM
// divides 20): in round r, warp w makes chunk TEAM r + w.  A chunk reads new
// words only from chunks at least seven before it, i.e. from earlier rounds,
// so one block barrier per round orders every such read after its write; a
// final barrier publishes the new block.  All TEAM warps call it.
template <typename OutT, int TEAM>
__device__ __forceinline__ void mt_twist_emit_team(const uint32_t *__restrict__ ob, uint32_t *__restrict__ nb, int warp,
                                                   int lane, OutT *o, uint32_t emit)
{
    static_assert(20 % TEAM == 0 && TEAM <= 4, "chunks per round");
#pragma unroll
    for (int r = 0; r < 20 / TEAM; ++r) {
        const int c = TEAM * r + warp;
        const int k = 32 * c + lane;
        if (k < kMtN) {
            const uint32_t a = ob[k];
            const uint32_t b = k + 1 < kMtN ? ob[k + 1] : nb[0];
            const uint32_t p = k < kMtN - kMtM ? ob[k + kMtM] : nb[k - (kMtN - kMtM)];
            const uint32_t x = mt_recur(a, b, p);
            nb[k] = x;
            if ((uint32_t)k < emit) o[k] = Cvt<OutT>::f(mt_temper(x));
        }
        __syncthreads();
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

// dst := the part of g(A) src that coefficients [c0, c1) of g contribute to
// result words [m0, m1), for one stream, by one warp (eq. (g_v)).  poly: g's
// 624 coefficient words, staged in shared memory by the caller.
//
// With src in window form x_0..x_623, A^i src is the window x_i..x_{i+623}, so
// result word m is the XOR of x_{i+m} over the set coefficients i of g.  Lane
// l owns W consecutive result words m = mbase + j (mbase = m0 + W l, clamped to
// m1 - W; a clamped lane writes only the words past the previous lane's) and
// keeps the W sequence words x_{i+mbase..i+mbase+W-1} in registers as a window
// that slides by one word per coefficient: one shared-memory load per
// coefficient, and W register XORs per set coefficient (one three-input XOR
// when two neighbouring coefficients are both set; W is even).  seq is this
// warp's 1248-word ring holding two consecutive 624-word blocks of the
// sequence (x at index i sits at seq[i mod 1248]): blocks 0 and 1 are made
// from src, and the warp twists on to the blocks around c0 before its first
// coefficient; block b then replaces block b - 2 at the first chunk of W
// coefficients from which no lane loads below index 624 (b - 1) again (loads
// from chunk start i0 on reach x_{i0+m0+W-1} and up).  c0 and c1 are multiples
// of W.  src and dst may be the same buffer only when every warp that reads
// src has copied it before any warp writes dst (sync: called between the two).
template <int W, typename Sync>
__device__ inline void mt_apply_poly_part(const uint32_t *__restrict__ poly, const uint32_t *src, uint32_t *dst,
                                          uint32_t *seq, int lane, int m0, int m1, int c0, int c1, Sync &&sync)
{
    static_assert(W % 2 == 0 && W <= 32, "pairs of coefficients per step");
    constexpr int RING = 2 * kMtN;
    const int mwant = m0 + W * lane;
    const int mbase = mwant + W <= m1 ? mwant : m1 - W;
    uint32_t acc[W], win[W];
#pragma unroll
    for (int j = 0; j < W; ++j) acc[j] = 0;
    mt_copy_state_warp(src, seq, lane);
    __syncwarp();
    sync();  // every warp holds its copy of src
    mt_twist_block(seq, seq + kMtN, lane);  // block 1 into slot 1
    const int b0 = c0 / kMtN;
    for (int b = 2; b <= b0 + 1; ++b) {  // blocks b0 and b0 + 1 in the ring
        __syncwarp();
        mt_twist_block(seq + ((b - 1) & 1) * kMtN, seq + (b & 1) * kMtN, lane);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < W - 1; ++j) win[j] = seq[(c0 + mbase + j) % RING];
    int next_block = b0 + 2;
    int p0 = (c0 + mbase + W - 1) % RING;  // ring position of the word loaded at step i0
    for (int i0 = c0; i0 < c1; i0 += W) {
        if (next_block <= 32 && i0 >= kMtN * (next_block - 1) - m0 - W + 1) {
            __syncwarp();
            mt_twist_block(seq + ((next_block - 1) & 1) * kMtN, seq + (next_block & 1) * kMtN, lane);
            ++next_block;
        }
        const int w = i0 >> 5, sh = i0 & 31;
        const uint64_t two = (uint64_t)poly[w] | ((uint64_t)(w + 1 < kMtPolyWords ? poly[w + 1] : 0u) << 32);
        const uint32_t bits = (uint32_t)(two >> sh) & (uint32_t)((1ull << W) - 1u);
#pragma unroll
        for (int u = 0; u < W; u += 2) {
            // step u: window slots (u + j) % W hold x_{i0+u+mbase+j}; the newest,
            // x_{i0+u+mbase+W-1}, goes into slot (u + W - 1) % W.  Step u + 1 needs
            // x_{i0+u+1+mbase+W-1} as its j = W - 1 word (nx); it replaces the
            // oldest word (slot u % W) only after both steps are applied.
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
    const int jfirst = mwant - mbase;  // words of this lane not already written by the previous lane
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (j >= jfirst) dst[mbase + j] = acc[j];
    __syncwarp();
}

constexpr int kMtChunkW = 20;                                       // result words per lane, coefficients per chunk
constexpr int kMtChunks = (kMtDeg + kMtChunkW - 1) / kMtChunkW;     // 997 chunks of coefficients

// dst := g(A) src for one stream by one warp (lane l owns 20 result words);
// poly in global memory, staged into pbuf (624 shared words of this warp).
__device__ inline void mt_apply_poly_warp(const uint32_t *__restrict__ poly, const uint32_t *src, uint32_t *dst,
                                          uint32_t *seq, uint32_t *pbuf, int lane)
{
    mt_copy_state_warp(poly, pbuf, lane);  // 624 words, as a state
    __syncwarp();
    mt_apply_poly_part<kMtChunkW>(pbuf, src, dst, seq, lane, 0, kMtN, 0, kMtChunkW * kMtChunks, [] {});
}

// The same by a team of T warps of one block (T = blockDim.x / 32), for one
// stream's latency: the coefficients are split in T consecutive ranges, warp w
// computes its range's contribution to all 624 result words into part[w]
// (T x 624 shared words), each warp making its own copy of the sequence up to
// its range, and the result is the XOR of the T parts (the sum of eq. (g_v) is
// linear over GF(2)).  The team stages the polynomial into pbuf (624 shared
// words) first; the block barrier after the copies of src lets dst alias src.
template <int T>
__device__ inline void mt_apply_poly_team(const uint32_t *__restrict__ poly, const uint32_t *src, uint32_t *dst,
                                          uint32_t *seq, uint32_t *pbuf, uint32_t *part, int warp, int lane)
{
    const int c0 = kMtChunkW * (kMtChunks * warp / T), c1 = kMtChunkW * (kMtChunks * (warp + 1) / T);
    for (int i = threadIdx.x; i < kMtPolyWords; i += 32 * T) pbuf[i] = poly[i];
    mt_apply_poly_part<kMtChunkW>(pbuf, src, T == 1 ? dst : part + warp * kMtN, seq, lane, 0, kMtN, c0, c1,
                                  [] { __syncthreads(); });
    __syncthreads();
    if constexpr (T > 1) {
        for (int m = threadIdx.x; m < kMtN; m += 32 * T) {
            uint32_t r = 0;
#pragma unroll
            for (int w = 0; w < T; ++w) r ^= part[w * kMtN + m];
            dst[m] = r;
        }
        __syncthreads();
    }
}

}  // namespace prand
