// Shared declarations of the batched persistent kernel (batch.cu) and the
// resident-stream server built on it (serve.cpp).
#pragma once

#include <vector>

#include "prand_internal.h"

namespace prand {

constexpr uint32_t kTileLast = 1u;      // the tile holds the request's last output: write the next state to wslot
constexpr uint32_t kTileVec = 2u;       // every row start is 16-byte aligned: vector / staged-row stores
constexpr uint32_t kTileFromSlot = 4u;  // start from the state in slot (else from the seeded base + stream * L)

// One unit of work for one warp (64 bytes).
struct BatchTile {
    uint64_t stream;  // stream index k (block splitting: base advanced by k L)
    uint64_t start;   // offset of the tile's first output inside the request
    uint64_t len;     // outputs in the tile
    uint64_t out;     // device address of the tile's first output
    uint32_t seclen;  // outputs per lane (MRG32K3A, LFSR113) or per lane group (GM/GQ)
    int32_t slot;     // state slot read with kTileFromSlot
    int32_t wslot;    // state slot written with kTileLast (a different buffer than slot)
    uint8_t gen, dtype;
    uint16_t flags;
    uint32_t req;     // index of the tile's request in its batch (completion tracking)
    uint32_t pad_[3];
};
static_assert(sizeof(BatchTile) == 64, "tile layout");

struct BatchCtx {
    const uint32_t *mrg_tab, *lfsr_tab, *mt_polys;
    const uint32_t *mt_win;                  // stream jumps by byte: [8][256][624] (digit 0 unused)
    const uint64_t *gm_tab[8];
    const void *base[PRAND_NUM_GENERATORS];  // base states of the batch's seed
    void *slots[PRAND_NUM_GENERATORS];       // resident-state arenas (server)
    uint32_t *tiles_left;                    // per request: tiles not finished (server), or null
    volatile uint32_t *done_list;            // mapped host memory: request index + 1, in completion order
    uint32_t *done_count;                    // device counter of done_list entries (zero at launch)
};

struct BatchParams {
    uint32_t seclen_mrg_lfsr = 8192;  // outputs per lane section (thread-per-section tiles), chosen by the tuner
    uint32_t seclen_gm = 8192;        // outputs per warp section (lane-per-point GM/GQ tiles)
    uint32_t block = 64;              // threads per block of the rest-of-generators build (64 or 128)
    uint32_t row_bytes = 128;         // its staged row size (128 or 256 bytes: 32 or 64 u32 outputs per row store)
};

prand_status_t batch_ctx(uint64_t seed, cudaStream_t st, BatchCtx *ctx, DevTables **T);
BatchParams batch_params();
void plan_request(const prand_request_t &r, int32_t slot, int32_t wslot, bool from_slot, const BatchParams &P,
                  std::vector<BatchTile> &out, uint32_t max_tiles = 0);
// Number of tiles plan_request() makes for r (without planning it).
uint64_t plan_tile_count(const prand_request_t &r, const BatchParams &P, uint32_t max_tiles = 0);
size_t slot_words(int gen);  // 32-bit words per state slot
prand_status_t upload_tiles(const std::vector<BatchTile> &tiles, cudaStream_t st, BatchTile **d_out, uint32_t **counter);
void order_tiles(std::vector<BatchTile> &tiles);
prand_status_t validate_requests(const prand_request_t *reqs, size_t n);
// A tile list runs in three parts, each a persistent launch of its own kernel
// build: [0, nmt) MT19937 tiles (many registers, shared memory), [nmt, nmt +
// nwide) the thread-per-stream GM/GQ tiles (GM55, GQ58.3, GQ58.4: their points
// need more registers than the last build allows), then every other generator
// (few registers, many resident warps).  order_tiles puts them in that order.
// With side branches (Branches), the MT19937 part and the thread-per-stream
// part each run on a branch stream of their own, forked from and joined back
// into `st`, so all three builds share the GPU at once; without them (the
// server's flights, one stream each) the parts run one after the other.
struct Branches {
    cudaStream_t st[2] = {};  // [0] MT19937 tiles, [1] thread-per-stream GM/GQ tiles
    cudaEvent_t fork[2] = {}, join[2] = {};
    prand_status_t create();
    void destroy();
};
bool wide_tile_gen(int gen);
uint32_t count_mt_tiles(const std::vector<BatchTile> &tiles);
uint32_t count_wide_tiles(const std::vector<BatchTile> &tiles, uint32_t nmt);
// Warps per MT19937 tile: the team applies each jump polynomial together
// (each warp takes a quarter of its coefficients) and then twists each output
// block together (five rounds of four 32-word chunks), for batches and the
// server alike (a batch of 10^4 mixed requests ran 16 % faster so than with
// one warp per tile).
constexpr int kMtTeam = 4;

prand_status_t launch_batch(const BatchTile *d_tiles, uint32_t ntiles, uint32_t nmt, uint32_t nwide,
                            uint32_t *d_counter, const BatchCtx &ctx, cudaStream_t st, const Branches *br = nullptr);

}  // namespace prand
