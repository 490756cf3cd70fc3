// Device side of the batched persistent launch (see batch.cu): the tile
// routines of each generator and the persistent kernel, templated on the
// kernel build (MODE), the block size and the staged row size, so that several
// translation units can instantiate different builds.
#pragma once

#include "batch.cuh"
#include "gm_impl.cuh"
#include "mrg_lfsr_dev.cuh"
#include "mt_dev.cuh"

namespace prand {

// Shared memory per warp: the largest of the MT19937 state pair (2 x 624 words),
// the staged row tile (32 rows of ROWB + 16 bytes) and the GM/GQ word slots.
constexpr int kWarpSmemBase = 5120;
template <int ROWB>
struct WarpSmem {
    static constexpr int bytes = RowFill<uint32_t, ROWB>::TILE > kWarpSmemBase ? RowFill<uint32_t, ROWB>::TILE : kWarpSmemBase;
};

// ------------------------------------------------------------------ MRG / LFSR tiles
template <typename OutT, int ROWB>
__device__ __forceinline__ void batch_mrg(const BatchTile &T, const BatchCtx &C, unsigned char *wsm, int lane)
{
    const uint64_t off = (uint64_t)lane * T.seclen;
    const uint64_t len = off < T.len ? min((uint64_t)T.seclen, T.len - off) : 0;
    uint32_t x[3], y[3];
    const bool from_slot = T.flags & kTileFromSlot;
    const uint32_t *src = from_slot ? (const uint32_t *)C.slots[PRAND_MRG32K3A] + 6 * (uint64_t)T.slot
                                    : (const uint32_t *)C.base[PRAND_MRG32K3A];
    for (int i = 0; i < 3; ++i) { x[i] = src[i]; y[i] = src[3 + i]; }
    if (len) {
        if (!from_slot)
            for (int b = 0; b < 64; ++b)
                if ((T.stream >> b) & 1u) mrg_apply_bit(C.mrg_tab, kMrgStreamShift + b, x, y);
        const uint64_t s = T.start + off;
        for (int b = 0; b < 64; ++b)
            if ((s >> b) & 1u) mrg_apply_bit(C.mrg_tab, b, x, y);
    }
    uint32_t x0 = x[0], x1 = x[1], x2 = x[2], y0 = y[0], y1 = y[1], y2 = y[2];
    OutT *o = (OutT *)T.out + off;
    if (T.flags & kTileVec) {
        fill_rows<OutT, ROWB>([&]() { return mrg_next(x0, x1, x2, y0, y1, y2); },
                        [](uint32_t u) { return Cvt<OutT, true>::f(u); }, o, len, wsm, lane);
    } else {
        for (uint64_t i = 0; i < len; ++i) o[i] = Cvt<OutT, true>::f(mrg_next(x0, x1, x2, y0, y1, y2));
    }
    if ((T.flags & kTileLast) && len && off + len == T.len) {
        uint32_t *d = (uint32_t *)C.slots[PRAND_MRG32K3A] + 6 * (uint64_t)T.wslot;
        d[0] = x0; d[1] = x1; d[2] = x2; d[3] = y0; d[4] = y1; d[5] = y2;
    }
}

template <typename OutT, int ROWB>
__device__ __forceinline__ void batch_lfsr(const BatchTile &T, const BatchCtx &C, unsigned char *wsm, int lane)
{
    const uint64_t off = (uint64_t)lane * T.seclen;
    const uint64_t len = off < T.len ? min((uint64_t)T.seclen, T.len - off) : 0;
    uint32_t z[4];
    const bool from_slot = T.flags & kTileFromSlot;
    const uint32_t *src = from_slot ? (const uint32_t *)C.slots[PRAND_LFSR113] + 4 * (uint64_t)T.slot
                                    : (const uint32_t *)C.base[PRAND_LFSR113];
    for (int c = 0; c < 4; ++c) z[c] = src[c];
    if (len) {
        // exponent (slot ? 0 : stream * 2^34) + start + off, as 128 bits
        const uint64_t s = T.start + off;
        uint64_t lo = s, hi = 0;
        if (!from_slot) {
            const uint64_t klo = T.stream << kLfsrStreamShift, khi = T.stream >> (64 - kLfsrStreamShift);
            lo = klo + s;
            hi = khi + (lo < klo ? 1u : 0u);
        }
        for (int b = 0; b < 64; ++b)
            if ((lo >> b) & 1u) lfsr_apply_bit(C.lfsr_tab, b, z);
        for (int b = 0; b < 64; ++b)
            if ((hi >> b) & 1u) lfsr_apply_bit(C.lfsr_tab, 64 + b, z);
    }
    uint32_t z0 = z[0], z1 = z[1], z2 = z[2], z3 = z[3];
    OutT *o = (OutT *)T.out + off;
    if (T.flags & kTileVec) {
        fill_rows<OutT, ROWB>([&]() { return lfsr_next(z0, z1, z2, z3); }, [](uint32_t u) { return Cvt<OutT>::f(u); }, o, len,
                        wsm, lane);
    } else {
        for (uint64_t i = 0; i < len; ++i) o[i] = Cvt<OutT>::f(lfsr_next(z0, z1, z2, z3));
    }
    if ((T.flags & kTileLast) && len && off + len == T.len) {
        uint32_t *d = (uint32_t *)C.slots[PRAND_LFSR113] + 4 * (uint64_t)T.wslot;
        d[0] = z0; d[1] = z1; d[2] = z2; d[3] = z3;
    }
}

// ------------------------------------------------------------------ GM / GQ tiles
// Lane-per-point ensembles (v = 1): the warp runs one section of the tile.
// Thread-per-stream ensembles (v = 3, 4): lane i runs section i of the tile,
// like the MRG32K3A and LFSR113 tiles.
template <int GEN, typename OutT>
__device__ __forceinline__ void batch_gm(const BatchTile &T, const BatchCtx &C, unsigned char *wsm, int lane)
{
    using P = GmT<GEN>;
    const uint64_t *tab = C.gm_tab[GEN - PRAND_GM19];
    const bool from_slot = T.flags & kTileFromSlot;
    const uint64_t *src = from_slot ? (const uint64_t *)C.slots[GEN] + 2 * P::s * (uint64_t)T.slot
                                    : (const uint64_t *)C.base[GEN];
    // exponent (slot ? 0 : stream * L) + start + off, as 128 bits
    auto exponent = [&](uint64_t off, uint64_t &lo, uint64_t &hi) {
        const uint64_t s = T.start + off;
        lo = s;
        hi = 0;
        if (!from_slot) {
            const uint64_t klo = T.stream * P::L_, khi = __umul64hi(T.stream, P::L_);
            lo = klo + s;
            hi = khi + (lo < klo ? 1u : 0u);
        }
    };
    if constexpr (P::lanes == 32) {
        const uint64_t len = min((uint64_t)T.seclen, T.len);
        if (len == 0) return;  // whole warp
        uint64_t zp = src[lane] >> P::t, zc = src[P::s + lane] >> P::t;
        uint64_t lo, hi;
        exponent(0, lo, hi);
        gm_jump128<GEN>(tab, lo, hi, zc, zp);
        OutT *o = (OutT *)T.out;
        uint32_t *myslot = reinterpret_cast<uint32_t *>(wsm) + 4 * lane;
        if (T.flags & kTileVec) gm_generate_section<GEN, OutT, true>(zc, zp, lane, o, len, myslot);
        else gm_generate_section<GEN, OutT, false>(zc, zp, lane, o, len, myslot);
        if ((T.flags & kTileLast) && len == T.len) {
            uint64_t *d = (uint64_t *)C.slots[GEN] + 2 * P::s * (uint64_t)T.wslot;
            d[lane] = zp << P::t;
            d[P::s + lane] = zc << P::t;
        }
    } else {
        using Z = GmZ<GEN>;
        const uint64_t off = (uint64_t)lane * T.seclen;
        const uint64_t len = off < T.len ? min((uint64_t)T.seclen, T.len - off) : 0;
        Z zc[P::s], zp[P::s];
        if (len) {
            uint64_t lo, hi;
            exponent(off, lo, hi);
            gmt_load<GEN>(tab, src, src + P::s, lo, hi, zc, zp);
        } else {
#pragma unroll
            for (int i = 0; i < P::s; ++i) { zc[i] = 0; zp[i] = 0; }
        }
        OutT *o = (OutT *)T.out + off;
        if (T.flags & kTileVec) {
            fill_rows<OutT, 128, true>([&]() { return gmt_next_word<GEN>(zc, zp); },
                                       [](uint32_t u) { return Cvt<OutT>::f(u); }, o, len, wsm, lane);
        } else {
            for (uint64_t i = 0; i < len; ++i) o[i] = Cvt<OutT>::f(gmt_next_word<GEN>(zc, zp));
        }
        if ((T.flags & kTileLast) && len && off + len == T.len) {
            uint64_t *d = (uint64_t *)C.slots[GEN] + 2 * P::s * (uint64_t)T.wslot;
            gmt_store<GEN>(zc, zp, d, d + P::s);
        }
    }
}

// ------------------------------------------------------------------ MT19937 tiles
// One tile = one request, run by a block of TEAM warps: the team applies the
// jump polynomials together (each warp takes a range of the coefficients),
// then makes the outputs together (batch_mt_emit_team).  Slot layout: 624 words of the current
// block, then the index inside it.  ring: the team's per-warp rings (2 x 624
// words each, warp w at ring + w * ring_stride words); tstate: 624 shared
// words holding the state between polynomial applications; pbuf: 624 shared
// words for the polynomial being applied; part: TEAM x 624 shared words for
// the warps' partial results.
// The outputs of an MT19937 tile made by the whole team: b0 holds the current
// block (written by warp 0), idx the position inside it.  Each further block
// is twisted by all TEAM warps (mt_twist_emit_team: TEAM chunks at a time
// instead of one), so a long request's sequential work shrinks by about TEAM.
template <typename OutT, int TEAM>
__device__ __forceinline__ void batch_mt_emit_team(const BatchTile &T, const BatchCtx &C, uint32_t *b0, uint32_t *b1,
                                                   uint32_t idx, int warp, int lane)
{
    __syncthreads();  // warp 0's copy of the current block is visible to the team
    OutT *o = (OutT *)T.out;
    const uint64_t nper = T.len;
    uint64_t done = 0;
    if (idx < (uint32_t)kMtN) {
        const uint32_t cnt = (uint32_t)min((uint64_t)(kMtN - idx), nper);
        for (uint32_t t = threadIdx.x; t < cnt; t += 32 * TEAM) o[t] = Cvt<OutT>::f(mt_temper(b0[idx + t]));
        done = cnt;
        idx += cnt;
    }
    bool in_b0 = true;
    while (done < nper) {
        const uint64_t rem = nper - done;
        const uint32_t emit = rem < (uint64_t)kMtN ? (uint32_t)rem : (uint32_t)kMtN;
        if (in_b0) mt_twist_emit_team<OutT, TEAM>(b0, b1, warp, lane, o + done, emit);
        else mt_twist_emit_team<OutT, TEAM>(b1, b0, warp, lane, o + done, emit);
        done += emit;
        idx = emit;
        in_b0 = !in_b0;
    }
    if ((T.flags & kTileLast) && warp == 0) {
        const uint32_t *cur = in_b0 ? b0 : b1;
        uint32_t *d = (uint32_t *)C.slots[PRAND_MT19937] + (kMtN + 1) * (uint64_t)T.wslot;
        mt_copy_state_warp(cur, d, lane);
        if (lane == 0) d[kMtN] = idx;
    }
    // every warp wrote outputs: each thread fences its own writes before the
    // block barrier after which one thread publishes the tile's completion
    __threadfence();
}

template <typename OutT, int TEAM>
__device__ __forceinline__ void batch_mt(const BatchTile &T, const BatchCtx &C, uint32_t *ring, int ring_stride,
                                         uint32_t *tstate, uint32_t *pbuf, uint32_t *part, int warp, int lane)
{
    uint32_t *b0 = ring, *b1 = ring + kMtN;  // warp 0's ring, for the outputs
    uint32_t idx = kMtN;
    if (T.flags & kTileFromSlot) {
        const uint32_t *src = (const uint32_t *)C.slots[PRAND_MT19937] + (kMtN + 1) * (uint64_t)T.slot;
        if (warp == 0) {
            mt_copy_state_warp(src, b0, lane);
            __syncwarp();
        }
        idx = src[kMtN];
    } else {
        // stream k = base advanced by k 2^432: one polynomial per nonzero byte of k
        const uint32_t *src = (const uint32_t *)C.base[PRAND_MT19937];
        bool first = true;
        for (int i = 0; i < kMtWinPositions; ++i) {
            const uint32_t d = (uint32_t)(T.stream >> (kMtWinBits * i)) & (uint32_t)(kMtWinDigits - 1);
            if (!d) continue;
            mt_apply_poly_team<TEAM>(C.mt_win + ((size_t)i * kMtWinDigits + d) * kMtPolyWords, first ? src : tstate, tstate,
                                     ring + warp * ring_stride, pbuf, part, warp, lane);
            first = false;
        }
        if (warp == 0) {
            mt_copy_state_warp(first ? src : tstate, b0, lane);
            __syncwarp();
        }
    }
    batch_mt_emit_team<OutT, TEAM>(T, C, b0, b1, idx, warp, lane);
}

// ------------------------------------------------------------------ the persistent kernels
// Three builds of the same loop: MT19937 tiles (jump chains that need many
// registers), the thread-per-stream GM/GQ tiles (8 or 12 points per lane, up
// to 128 registers), and every other generator (48 registers, so many more
// resident warps).  A batch's tiles come in that order (order_tiles).
enum { kModeMt = 0, kModeRest = 1, kModeWide = 2 };
constexpr int kModes = 3;

template <typename OutT, int MODE, int ROWB>
__device__ __forceinline__ void batch_tile(const BatchTile &T, const BatchCtx &C, unsigned char *wsm, int lane)
{
    if constexpr (MODE == kModeWide) {
        switch (T.gen) {
        case PRAND_GM55: batch_gm<PRAND_GM55, OutT>(T, C, wsm, lane); break;
        case PRAND_GQ58_3: batch_gm<PRAND_GQ58_3, OutT>(T, C, wsm, lane); break;
        case PRAND_GQ58_4: batch_gm<PRAND_GQ58_4, OutT>(T, C, wsm, lane); break;
        default: break;  // not a tile of this build (the host partitions the list)
        }
    } else {
        switch (T.gen) {
        case PRAND_MRG32K3A: batch_mrg<OutT, ROWB>(T, C, wsm, lane); break;
        case PRAND_LFSR113: batch_lfsr<OutT, ROWB>(T, C, wsm, lane); break;
        case PRAND_GM19: batch_gm<PRAND_GM19, OutT>(T, C, wsm, lane); break;
        case PRAND_GM29: batch_gm<PRAND_GM29, OutT>(T, C, wsm, lane); break;
        case PRAND_GM31: batch_gm<PRAND_GM31, OutT>(T, C, wsm, lane); break;
        case PRAND_GM61: batch_gm<PRAND_GM61, OutT>(T, C, wsm, lane); break;
        case PRAND_GQ58_1: batch_gm<PRAND_GQ58_1, OutT>(T, C, wsm, lane); break;
        default: break;  // not a tile of this build (the host partitions the list)
        }
    }
}

// Completion of a request: the request's last tile to finish publishes it.
// Every tile fences its writes before counting down; the last one fences to
// system scope and appends the request to the host-visible list.
__device__ __forceinline__ void batch_tile_done(const BatchTile &T, const BatchCtx &ctx)
{
    if (!ctx.tiles_left) return;
    __threadfence();
    if (atomicSub(&ctx.tiles_left[T.req], 1u) == 1u) {
        __threadfence_system();
        const uint32_t slot = atomicAdd(ctx.done_count, 1u);
        ctx.done_list[slot] = T.req + 1u;
    }
}

// BS threads per block; the builds aim at the resident warps their registers
// allow (the rest: 40 warps per SM at 48 registers; thread-per-stream GM/GQ:
// 16 warps at 128; MT19937: whatever its jump chains need).  ROWB: the staged
// row size of the thread-per-section tiles (MRG32K3A, LFSR113).  The MT19937
// build claims tiles per block (a team of BS / 32 warps per tile), the others
// per warp.
template <int MODE, int BS, int ROWB>
__global__ void __launch_bounds__(BS, (MODE == kModeRest ? 1280 / BS : MODE == kModeWide ? 512 / BS : 1)) batch_kernel(
    const BatchTile *__restrict__ tiles, uint32_t ntiles, uint32_t *counter, BatchCtx ctx)
{
    __shared__ __align__(16) unsigned char smem[BS / 32][WarpSmem<ROWB>::bytes];
    if constexpr (MODE == kModeMt) {
        constexpr int TEAM = BS / 32;  // one team of warps per block
        static_assert(TEAM == kMtTeam, "MT19937 build: one team of warps per tile");
        __shared__ uint32_t tstate[kMtN];
        __shared__ uint32_t pbuf[kMtPolyWords];
        __shared__ uint32_t part[TEAM > 1 ? TEAM * kMtN : 1];
        __shared__ uint32_t claimed;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (;;) {
            if (threadIdx.x == 0) claimed = atomicAdd(counter, 1u);
            __syncthreads();
            const uint32_t t = claimed;
            __syncthreads();
            if (t >= ntiles) return;
            const BatchTile T = tiles[t];
            uint32_t *ring = reinterpret_cast<uint32_t *>(&smem[0][0]);
            constexpr int stride = WarpSmem<ROWB>::bytes / 4;
            if (T.dtype == PRAND_DTYPE_U32) batch_mt<uint32_t, TEAM>(T, ctx, ring, stride, tstate, pbuf, part, warp, lane);
            else if (T.dtype == PRAND_DTYPE_F32) batch_mt<float, TEAM>(T, ctx, ring, stride, tstate, pbuf, part, warp, lane);
            else batch_mt<double, TEAM>(T, ctx, ring, stride, tstate, pbuf, part, warp, lane);
            __syncthreads();
            if (threadIdx.x == 0) batch_tile_done(T, ctx);
        }
    } else {
        const int lane = threadIdx.x & 31;
        unsigned char *wsm = smem[threadIdx.x >> 5];
        for (;;) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(counter, 1u);
            t = __shfl_sync(kFull, t, 0);
            if (t >= ntiles) return;
            const BatchTile T = tiles[t];
            if (T.dtype == PRAND_DTYPE_U32) batch_tile<uint32_t, MODE, ROWB>(T, ctx, wsm, lane);
            else if (T.dtype == PRAND_DTYPE_F32) batch_tile<float, MODE, ROWB>(T, ctx, wsm, lane);
            else batch_tile<double, MODE, ROWB>(T, ctx, wsm, lane);
            __syncwarp();
            if (lane == 0) batch_tile_done(T, ctx);
            __syncwarp();
        }
    }
}

// Builds of the rest-of-generators kernel by (threads per block, row bytes),
// variant index 2 (BS == 128) + (ROWB == 256).
constexpr int kRestVariants = 4;
inline int rest_variant(uint32_t block, uint32_t row_bytes) { return 2 * (block == 128) + (row_bytes == 256); }
inline uint32_t rest_block(int variant) { return variant >= 2 ? 128 : 64; }
// (batch_rest_64.cu: variants 0 and 1; batch_rest_128.cu: 2 and 3; row256 selects ROWB)
int rest_blocks_per_sm_64(bool row256);
int rest_blocks_per_sm_128(bool row256);
void rest_launch_64(bool row256, unsigned grid, cudaStream_t st, const BatchTile *tiles, uint32_t ntiles,
                    uint32_t *counter, const BatchCtx &ctx);
void rest_launch_128(bool row256, unsigned grid, cudaStream_t st, const BatchTile *tiles, uint32_t ntiles,
                     uint32_t *counter, const BatchCtx &ctx);
inline int rest_blocks_per_sm(int v) { return v >= 2 ? rest_blocks_per_sm_128(v & 1) : rest_blocks_per_sm_64(v & 1); }
inline void rest_launch(int v, unsigned grid, cudaStream_t st, const BatchTile *tiles, uint32_t ntiles,
                        uint32_t *counter, const BatchCtx &ctx)
{
    if (v >= 2) rest_launch_128(v & 1, grid, st, tiles, ntiles, counter, ctx);
    else rest_launch_64(v & 1, grid, st, tiles, ntiles, counter, ctx);
}

}  // namespace prand
