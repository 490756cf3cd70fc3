// Batched generation: thousands of requests (generator, stream index, length,
// element type, output pointer) of mixed generators and uneven lengths in one
// persistent launch, with each request's jump-ahead (block splitting, Table 4,
// plus the offset of its section) fused in front of its generation.
//
// Work unit: a tile, run by one warp.  MRG32K3A / LFSR113 tiles are up to 32
// sections of one request (one lane each, rows written through the staged
// 128-byte row stores); GM/GQ tiles are up to 32 / lanes sections (one lane
// group each); MT19937 tiles are one whole request (the jump is a chain of
// polynomial applications by the warp, Sec. 5.4).  Warps claim tiles from an
// atomic counter, so short and long tiles balance across the GPU; tiles are
// ordered longest first.
//
// The same kernel serves the resident-stream server: a tile may start from a
// state slot instead of the seeded base, and the tile that ends a request
// writes the stream's next state back to its slot.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "batch_kernel.cuh"

namespace prand {

constexpr int kBatchThreads = 64;  // the wide build: small blocks (a warp on a long tile holds little besides itself)

// One MT19937 stream for the per-request form: stream k = base advanced by
// k 2^432, one window polynomial per nonzero byte of k (the same jump the
// batched MT19937 tiles take), by one warp.
__global__ void __launch_bounds__(32) mt_window_init_kernel(const uint32_t *base, const uint32_t *win, uint64_t k,
                                                            uint32_t *dst)
{
    __shared__ uint32_t seq[2 * kMtN], pbuf[kMtPolyWords];
    const int lane = threadIdx.x;
    bool first = true;
    for (int i = 0; i < kMtWinPositions; ++i) {
        const uint32_t d = (uint32_t)(k >> (kMtWinBits * i)) & (uint32_t)(kMtWinDigits - 1);
        if (!d) continue;
        mt_apply_poly_warp(win + ((size_t)i * kMtWinDigits + d) * kMtPolyWords, first ? base : dst, dst, seq, pbuf,
                           lane);
        first = false;
        __syncwarp();
    }
    if (first) mt_copy_state_warp(base, dst, lane);
}


// ------------------------------------------------------------------ host: engine
namespace {

size_t esize(int dtype) { return dtype == PRAND_DTYPE_F64 ? 8 : 4; }

struct SeedBases {
    uint64_t seed = 0;
    void *dev = nullptr;
    size_t off[PRAND_NUM_GENERATORS] = {};
};

struct Engine {
    int device = -1;
    DevTables *T = nullptr;
    std::vector<SeedBases> bases;  // small cache, most recent last
    BatchTile *d_tiles = nullptr;
    size_t d_cap = 0;
    BatchTile *h_tiles = nullptr;  // pinned staging
    size_t h_cap = 0;
    cudaEvent_t staged = nullptr;  // the last copy out of h_tiles
    uint32_t *d_counter = nullptr;
    BatchParams params;
    int sms = 1, blocks_per_sm[kModes] = { 1, 1, 1 };  // the wide build's (the others keep their own)
    int mt_team_bps = 1;                               // MT19937 build: a team of warps per tile
    int rest_bps[kRestVariants] = { 1, 1, 1, 1 };      // the rest build's variants
    Branches br;                                  // side branches of mixed launches
    std::mutex aux_mu;
    bool ready = false;
};

constexpr int kMaxDev = 64;
Engine g_eng[kMaxDev];
std::mutex g_eng_mu;

prand_status_t engine_get(Engine **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return PRAND_ERR_CUDA;
    Engine &E = g_eng[dev];
    if (!E.ready) {
        E.device = dev;
        prand_status_t s = get_tables(PRAND_MT19937, &E.T);
        if (s != PRAND_OK) return s;
        if (!dev_alloc(&E.d_counter, 64)) return PRAND_ERR_NOMEM;
        if (cudaEventCreateWithFlags(&E.staged, cudaEventDisableTiming) != cudaSuccess) return PRAND_ERR_CUDA;
        E.sms = device_sm_count();
        {
            int bps = 0;
            const cudaError_t e =
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel<kModeWide, kBatchThreads, 128>, kBatchThreads, 0);
            E.blocks_per_sm[kModeWide] = (e == cudaSuccess && bps >= 1) ? bps : 1;
        }
        for (int v = 0; v < kRestVariants; ++v) E.rest_bps[v] = rest_blocks_per_sm(v);
        {
            int bps = 0;
            const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &bps, batch_kernel<kModeMt, 32 * kMtTeam, 128>, 32 * kMtTeam, 0);
            E.mt_team_bps = (e == cudaSuccess && bps >= 1) ? bps : 1;
        }
        if (E.br.create() != PRAND_OK) return PRAND_ERR_CUDA;
        const char *path = getenv("PRAND_TUNE_CACHE");
        if (path) {
            FILE *f = fopen(path, "r");
            if (f) {
                unsigned a = 0, b = 0, c = 0, d = 0;
                if (fscanf(f, "{\"seclen_mrg_lfsr\": %u, \"seclen_gm\": %u, \"block\": %u, \"row_bytes\": %u", &a, &b,
                           &c, &d) == 4 && a && b && a % 4 == 0 && b % 4 == 0 && (c == 64 || c == 128) &&
                    (d == 128 || d == 256)) {
                    E.params.seclen_mrg_lfsr = a;
                    E.params.seclen_gm = b;
                    E.params.block = c;
                    E.params.row_bytes = d;
                }
                fclose(f);
            }
        }
        E.ready = true;
    }
    *out = &E;
    return PRAND_OK;
}

// Base states of all eleven generators for one seed (computed on the device).
prand_status_t engine_bases(Engine &E, uint64_t seed, cudaStream_t st, const SeedBases **out)
{
    for (size_t i = 0; i < E.bases.size(); ++i)
        if (E.bases[i].seed == seed) { *out = &E.bases[i]; return PRAND_OK; }
    SeedBases B;
    B.seed = seed;
    size_t total = 0;
    for (int g = 0; g < PRAND_NUM_GENERATORS; ++g) {
        B.off[g] = total;
        total += (state_bytes_per_stream(g) + 255) & ~(size_t)255;
    }
    if (!dev_alloc(&B.dev, total)) return PRAND_ERR_NOMEM;
    prand_status_t s = PRAND_OK;
    for (int g = 0; g < PRAND_NUM_GENERATORS && s == PRAND_OK; ++g) {
        void *p = (char *)B.dev + B.off[g];
        if (g == PRAND_MT19937) s = mt_seed(seed, p, st);
        else if (is_gm(g)) { Variant V; variant_params(g, 0, &V); s = gm_seed(g, E.T, seed, V, p, st); }
        else s = mrg_lfsr_seed(g, seed, p, st);
    }
    // wait once, so later batches on any stream see the bases
    if (s == PRAND_OK && cudaStreamSynchronize(st) != cudaSuccess) s = PRAND_ERR_CUDA;
    if (s != PRAND_OK) { cudaFree(B.dev); return s; }
    if (E.bases.size() >= 4) {
        cudaStreamSynchronize(st);
        cudaFree(E.bases.front().dev);
        E.bases.erase(E.bases.begin());
    }
    E.bases.push_back(B);
    *out = &E.bases.back();
    return PRAND_OK;
}

}  // namespace

prand_status_t batch_ctx(uint64_t seed, cudaStream_t st, BatchCtx *ctx, DevTables **T)
{
    Engine *E;
    prand_status_t s = engine_get(&E);
    if (s != PRAND_OK) return s;
    const SeedBases *B;
    if ((s = engine_bases(*E, seed, st, &B)) != PRAND_OK) return s;
    memset(ctx, 0, sizeof *ctx);
    ctx->mrg_tab = E->T->mrg;
    ctx->lfsr_tab = E->T->lfsr;
    ctx->mt_polys = E->T->mt;
    if ((s = get_mt_window(E->T)) != PRAND_OK) return s;
    ctx->mt_win = E->T->mt_win;
    for (int g = 0; g < 8; ++g) ctx->gm_tab[g] = E->T->gm[g];
    for (int g = 0; g < PRAND_NUM_GENERATORS; ++g) ctx->base[g] = (const char *)B->dev + B->off[g];
    if (T) *T = E->T;
    return PRAND_OK;
}

BatchParams batch_params()
{
    Engine *E;
    if (engine_get(&E) != PRAND_OK) return BatchParams();
    return E->params;
}

// Split one request into tiles (appended to `out`).  from_slot: continue the
// state in `slot`; else start from the seeded base advanced to the request's
// stream.  wslot >= 0: the request's last tile writes the next state there.
// Section length (outputs per lane) of r's tiles: the tuned default, made
// longer for long requests so that r yields at most max_tiles tiles (a
// multiple of 128 outputs).
static uint64_t section_length(const prand_request_t &r, const BatchParams &P, uint32_t max_tiles)
{
    const uint64_t lanes_per_tile = is_gm(r.gen) ? (uint64_t)(32 / gm_params(r.gen).lanes) : 32ull;
    // one section per warp (lane-per-point GM/GQ) or one per lane (the rest)
    uint64_t sec = lanes_per_tile == 1 ? P.seclen_gm : P.seclen_mrg_lfsr;
    if (max_tiles) {
        const uint64_t need = (r.length + lanes_per_tile * max_tiles - 1) / (lanes_per_tile * max_tiles);
        if (need > sec) sec = (need + 127) & ~127ull;
    }
    return sec;
}

uint64_t plan_tile_count(const prand_request_t &r, const BatchParams &P, uint32_t max_tiles)
{
    if (r.length == 0) return 0;
    if (r.gen == PRAND_MT19937) return 1;
    const uint64_t lanes_per_tile = is_gm(r.gen) ? (uint64_t)(32 / gm_params(r.gen).lanes) : 32ull;
    const uint64_t per_tile = section_length(r, P, max_tiles) * lanes_per_tile;
    return (r.length + per_tile - 1) / per_tile;
}

void plan_request(const prand_request_t &r, int32_t slot, int32_t wslot, bool from_slot, const BatchParams &P,
                  std::vector<BatchTile> &out, uint32_t max_tiles)
{
    if (r.length == 0) return;
    const int gen = r.gen;
    const size_t es = esize(r.dtype);
    const uintptr_t base = (uintptr_t)r.dev_out;
    auto vec_ok = [&](uint64_t seclen) { return base % 16 == 0 && (seclen * es) % 16 == 0 && seclen % 4 == 0; };
    const uint16_t fs = from_slot ? (uint16_t)kTileFromSlot : (uint16_t)0;
    if (gen == PRAND_MT19937) {
        BatchTile t = {};
        t.stream = r.stream; t.start = 0; t.len = r.length; t.out = base;
        t.seclen = 0; t.gen = (uint8_t)gen; t.dtype = (uint8_t)r.dtype; t.slot = slot; t.wslot = wslot;
        t.flags = (uint16_t)(fs | (wslot >= 0 ? kTileLast : 0u));
        out.push_back(t);
        return;
    }
    const uint64_t lanes_per_tile = is_gm(gen) ? (uint64_t)(32 / gm_params(gen).lanes) : 32ull;
    const uint64_t sec = section_length(r, P, max_tiles);
    const uint64_t per_tile = sec * lanes_per_tile;
    for (uint64_t off = 0; off < r.length; off += per_tile) {
        BatchTile t = {};
        t.stream = r.stream; t.start = off; t.len = std::min(per_tile, r.length - off);
        t.out = base + off * es;
        t.seclen = (uint32_t)sec; t.gen = (uint8_t)gen; t.dtype = (uint8_t)r.dtype; t.slot = slot; t.wslot = wslot;
        t.flags = (uint16_t)(fs | (vec_ok(sec) ? kTileVec : 0u) |
                             ((wslot >= 0 && off + t.len == r.length) ? kTileLast : 0u));
        out.push_back(t);
    }
}

size_t slot_words(int gen)
{
    if (gen == PRAND_MT19937) return kMtN + 1;
    return state_bytes_per_stream(gen) / 4;
}

bool wide_tile_gen(int gen) { return is_gm(gen) && gm_params(gen).lanes == 1; }

// MT19937 tiles first, then the thread-per-stream GM/GQ tiles, then the rest;
// longest first within each part (MT19937 jump chains are the longest).
static uint64_t tile_cost(const BatchTile &t)
{
    if (t.gen == PRAND_MT19937) return (1ull << 41) + t.len;
    if (wide_tile_gen(t.gen)) return (1ull << 40) + t.len;
    return t.len / (t.gen == PRAND_MRG32K3A || t.gen == PRAND_LFSR113 ? 32 : 1);
}

void order_tiles(std::vector<BatchTile> &tiles)
{
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const BatchTile &a, const BatchTile &b) { return tile_cost(a) > tile_cost(b); });
}

prand_status_t validate_requests(const prand_request_t *reqs, size_t n)
{
    if (!reqs && n) return PRAND_ERR_ARG;
    for (size_t i = 0; i < n; ++i) {
        const prand_request_t &r = reqs[i];
        if (r.gen < 0 || r.gen >= PRAND_NUM_GENERATORS || r.dtype < 0 || r.dtype > 2) return PRAND_ERR_ARG;
        if (r.length && !r.dev_out) return PRAND_ERR_ARG;
        if ((uintptr_t)r.dev_out % esize(r.dtype)) return PRAND_ERR_ALIGN;
        uint64_t bytes;
        if (__builtin_mul_overflow(r.length, (uint64_t)esize(r.dtype), &bytes)) return PRAND_ERR_ARG;
    }
    return PRAND_OK;
}

// Persistent grid of a build: enough blocks for the tiles, at most the
// resident blocks of the whole GPU.
static unsigned batch_grid(uint32_t ntiles, uint32_t block, int blocks_per_sm)
{
    Engine *E;
    if (engine_get(&E) != PRAND_OK) return 1;
    uint64_t warps_needed = ntiles, per_block = block / 32;
    uint64_t g = std::min<uint64_t>((warps_needed + per_block - 1) / per_block, (uint64_t)E->sms * blocks_per_sm);
    return (unsigned)std::max<uint64_t>(g, 1);
}

uint32_t count_mt_tiles(const std::vector<BatchTile> &tiles)
{
    uint32_t n = 0;
    while (n < tiles.size() && tiles[n].gen == PRAND_MT19937) ++n;
    return n;
}

uint32_t count_wide_tiles(const std::vector<BatchTile> &tiles, uint32_t nmt)
{
    uint32_t n = 0;
    while (nmt + n < tiles.size() && wide_tile_gen(tiles[nmt + n].gen)) ++n;
    return n;
}

// Tiles [0, nmt): MT19937 (counter[0]); [nmt, nmt + nwide): thread-per-stream
// GM/GQ (counter[2]); the rest (counter[1]).  With MT19937 tiles beside others
// with side branches the MT19937 part runs on br->st[0] and the
// thread-per-stream part on br->st[1], each forked from and joined back into `st`.
prand_status_t Branches::create()
{
    for (int b = 0; b < 2; ++b)
        if (cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming) != cudaSuccess)
            return PRAND_ERR_CUDA;
    return PRAND_OK;
}

void Branches::destroy()
{
    for (int b = 0; b < 2; ++b) {
        if (st[b]) cudaStreamDestroy(st[b]);
        if (fork[b]) cudaEventDestroy(fork[b]);
        if (join[b]) cudaEventDestroy(join[b]);
        st[b] = nullptr;
        fork[b] = join[b] = nullptr;
    }
}

prand_status_t launch_batch(const BatchTile *d_tiles, uint32_t ntiles, uint32_t nmt, uint32_t nwide,
                            uint32_t *d_counter, const BatchCtx &ctx, cudaStream_t st, const Branches *br)
{
    if (cudaMemsetAsync(d_counter, 0, 3 * sizeof(uint32_t), st) != cudaSuccess) return PRAND_ERR_CUDA;
    if (!ntiles) return PRAND_OK;
    const uint32_t nrest = ntiles - nmt - nwide;
    // a part goes to its branch when another part runs beside it
    const bool on_branch[2] = { br && nmt && (nwide || nrest), br && nwide && nrest };
    prand_status_t s = PRAND_OK;
    for (int b = 0; b < 2; ++b)
        if (on_branch[b] && (cudaEventRecord(br->fork[b], st) != cudaSuccess ||
                             cudaStreamWaitEvent(br->st[b], br->fork[b], 0) != cudaSuccess))
            return PRAND_ERR_CUDA;
    Engine *E;
    if ((s = engine_get(&E)) != PRAND_OK) return s;
    if (nmt) {
        cudaStream_t ms = on_branch[0] ? br->st[0] : st;
        const unsigned g = batch_grid(nmt, 32, E->mt_team_bps);  // one tile per block
        batch_kernel<kModeMt, 32 * kMtTeam, 128><<<g, 32 * kMtTeam, 0, ms>>>(d_tiles, nmt, d_counter, ctx);
        if ((s = launch_check()) != PRAND_OK) return s;
    }
    if (nwide) {
        const unsigned g = batch_grid(nwide, kBatchThreads, E->blocks_per_sm[kModeWide]);
        batch_kernel<kModeWide, kBatchThreads, 128><<<g, kBatchThreads, 0, on_branch[1] ? br->st[1] : st>>>(
            d_tiles + nmt, nwide, d_counter + 2, ctx);
        if ((s = launch_check()) != PRAND_OK) return s;
    }
    if (nrest) {
        const int v = rest_variant(E->params.block, E->params.row_bytes);
        rest_launch(v, batch_grid(nrest, rest_block(v), E->rest_bps[v]), st, d_tiles + nmt + nwide, nrest,
                    d_counter + 1, ctx);
        if ((s = launch_check()) != PRAND_OK) return s;
    }
    for (int b = 0; b < 2; ++b)
        if (on_branch[b] && (cudaEventRecord(br->join[b], br->st[b]) != cudaSuccess ||
                             cudaStreamWaitEvent(st, br->join[b], 0) != cudaSuccess))
            return PRAND_ERR_CUDA;
    return PRAND_OK;
}

prand_status_t upload_tiles(const std::vector<BatchTile> &tiles, cudaStream_t st, BatchTile **d_out, uint32_t **counter)
{
    Engine *E;
    prand_status_t s = engine_get(&E);
    if (s != PRAND_OK) return s;
    const size_t n = tiles.size();
    if (cudaEventSynchronize(E->staged) != cudaSuccess) return PRAND_ERR_CUDA;  // staging free again
    if (n > E->h_cap) {
        if (E->h_tiles) cudaFreeHost(E->h_tiles);
        E->h_cap = std::max<size_t>(n, 2 * E->h_cap);
        if (!host_alloc(&E->h_tiles, E->h_cap * sizeof(BatchTile))) { E->h_cap = 0; E->h_tiles = nullptr; return PRAND_ERR_NOMEM; }
    }
    if (n > E->d_cap) {
        // the previous batch may still read the old buffer: free it in stream order
        if (E->d_tiles) { cudaStreamSynchronize(st); cudaFree(E->d_tiles); }
        E->d_cap = std::max<size_t>(n, 2 * E->d_cap);
        if (!dev_alloc(&E->d_tiles, E->d_cap * sizeof(BatchTile))) { E->d_cap = 0; E->d_tiles = nullptr; return PRAND_ERR_NOMEM; }
    }
    if (n) {
        memcpy(E->h_tiles, tiles.data(), n * sizeof(BatchTile));
        if (cudaMemcpyAsync(E->d_tiles, E->h_tiles, n * sizeof(BatchTile), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return PRAND_ERR_CUDA;
        if (cudaEventRecord(E->staged, st) != cudaSuccess) return PRAND_ERR_CUDA;
    }
    *d_out = E->d_tiles;
    *counter = E->d_counter;
    return PRAND_OK;
}

}  // namespace prand

using namespace prand;

// ------------------------------------------------------------------ C ABI
struct prand_batch_plan_s {
    int device = -1;
    BatchTile *d_tiles = nullptr;
    uint32_t ntiles = 0, nmt = 0, nwide = 0;
    Branches br;  // the side branches while capturing
    uint32_t *d_counter = nullptr;
    BatchCtx ctx;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

prand_status_t prand_batch_run(const prand_request_t *reqs, size_t n, uint64_t seed, prand_stream_t stream)
{
    prand_status_t s = validate_requests(reqs, n);
    if (s != PRAND_OK || n == 0) return s;
    cudaStream_t st = (cudaStream_t)stream;
    BatchCtx ctx;
    if ((s = batch_ctx(seed, st, &ctx, nullptr)) != PRAND_OK) return s;
    const BatchParams P = batch_params();
    std::vector<BatchTile> tiles;
    tiles.reserve(n * 2);
    for (size_t i = 0; i < n; ++i) plan_request(reqs[i], -1, -1, false, P, tiles);
    order_tiles(tiles);
    if (tiles.size() > 0xFFFFFFFFull) return PRAND_ERR_ARG;
    BatchTile *d_tiles;
    uint32_t *counter;
    if ((s = upload_tiles(tiles, st, &d_tiles, &counter)) != PRAND_OK) return s;
    Engine *E;
    if ((s = engine_get(&E)) != PRAND_OK) return s;
    std::lock_guard<std::mutex> lk(E->aux_mu);  // one user of the branches at a time
    const uint32_t nmt = count_mt_tiles(tiles);
    return launch_batch(d_tiles, (uint32_t)tiles.size(), nmt, count_wide_tiles(tiles, nmt), counter, ctx, st, &E->br);
}

prand_status_t prand_batch_plan_create(prand_batch_plan_t *out, const prand_request_t *reqs, size_t n, uint64_t seed)
{
    if (!out) return PRAND_ERR_ARG;
    *out = nullptr;
    prand_status_t s = validate_requests(reqs, n);
    if (s != PRAND_OK) return s;
    prand_batch_plan_t p = new (std::nothrow) prand_batch_plan_s;
    if (!p) return PRAND_ERR_NOMEM;
    cudaGetDevice(&p->device);
    cudaStream_t cap = nullptr;
    auto fail = [&](prand_status_t e) {
        if (cap) cudaStreamDestroy(cap);
        p->br.destroy();
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        if (p->d_tiles) cudaFree(p->d_tiles);
        if (p->d_counter) cudaFree(p->d_counter);
        delete p;
        return e;
    };
    if ((s = batch_ctx(seed, 0, &p->ctx, nullptr)) != PRAND_OK) return fail(s);
    const BatchParams P = batch_params();
    std::vector<BatchTile> tiles;
    for (size_t i = 0; i < n; ++i) plan_request(reqs[i], -1, -1, false, P, tiles);
    order_tiles(tiles);
    if (tiles.size() > 0xFFFFFFFFull) return fail(PRAND_ERR_ARG);
    p->ntiles = (uint32_t)tiles.size();
    p->nmt = count_mt_tiles(tiles);
    p->nwide = count_wide_tiles(tiles, p->nmt);
    if (!dev_alloc(&p->d_counter, 64)) return fail(PRAND_ERR_NOMEM);
    if (p->br.create() != PRAND_OK) return fail(PRAND_ERR_CUDA);
    if (p->ntiles) {
        if (!dev_alloc(&p->d_tiles, tiles.size() * sizeof(BatchTile))) return fail(PRAND_ERR_NOMEM);
        if (cudaMemcpy(p->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(PRAND_ERR_CUDA);
    }
    if (cudaStreamSynchronize(0) != cudaSuccess) return fail(PRAND_ERR_CUDA);
    // capture: counter reset + the persistent launches (the MT19937 and
    // thread-per-stream parts forked onto the plan's branch streams and joined back)
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return fail(PRAND_ERR_CUDA);
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(PRAND_ERR_CUDA);
    prand_status_t ls = launch_batch(p->d_tiles, p->ntiles, p->nmt, p->nwide, p->d_counter, p->ctx, cap, &p->br);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cap, &g);
    p->graph = g;
    if (ls != PRAND_OK || ce != cudaSuccess) return fail(PRAND_ERR_CUDA);
    if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) return fail(PRAND_ERR_CUDA);
    cudaStreamDestroy(cap);
    cap = nullptr;
    *out = p;
    return PRAND_OK;
}

prand_status_t prand_batch_plan_launch(prand_batch_plan_t p, prand_stream_t stream)
{
    if (!p || !p->exec) return PRAND_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return PRAND_ERR_STATE;
    g_launches.fetch_add(p->ntiles ? 1 : 0, std::memory_order_relaxed);
    return cudaGraphLaunch(p->exec, (cudaStream_t)stream) == cudaSuccess ? PRAND_OK : PRAND_ERR_CUDA;
}

prand_status_t prand_batch_plan_destroy(prand_batch_plan_t p)
{
    if (!p) return PRAND_OK;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_tiles) cudaFree(p->d_tiles);
    if (p->d_counter) cudaFree(p->d_counter);
    p->br.destroy();
    delete p;
    return PRAND_OK;
}

prand_status_t prand_batch_autotune(const prand_request_t *reqs, size_t n, uint64_t seed, prand_stream_t stream,
                                    uint32_t *seclen_mrg_lfsr, uint32_t *seclen_gm, uint32_t *block,
                                    uint32_t *row_bytes, float *best_ms)
{
    prand_status_t s = validate_requests(reqs, n);
    if (s != PRAND_OK) return s;
    Engine *E;
    if ((s = engine_get(&E)) != PRAND_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const BatchParams keep = E->params;
    BatchParams best = keep;
    float best_t = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one candidate: a graph plan with these parameters, one warm-up launch,
    // the mean of three timed launches
    auto try_params = [&](const BatchParams &c) {
        E->params = c;
        prand_batch_plan_t plan;
        if ((s = prand_batch_plan_create(&plan, reqs, n, seed)) != PRAND_OK) return;
        prand_batch_plan_launch(plan, stream);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) prand_batch_plan_launch(plan, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3;
        prand_batch_plan_destroy(plan);
        if (ms < best_t) { best_t = ms; best = c; }
    };
    // coordinate search: the two section lengths (outputs per lane and per
    // warp section), then the rest build's threads per block and staged row
    // size (outputs per row store) at the best lengths
    const uint32_t cand[] = { 2048, 8192, 32768 };
    for (uint32_t a : cand)
        for (uint32_t b : cand) {
            if (s != PRAND_OK) break;
            BatchParams c = keep;
            c.seclen_mrg_lfsr = a;
            c.seclen_gm = b;
            try_params(c);
        }
    const BatchParams lengths = best;
    for (uint32_t bs : { 64u, 128u })
        for (uint32_t rb : { 128u, 256u }) {
            if (s != PRAND_OK) break;
            BatchParams c = lengths;
            c.block = bs;
            c.row_bytes = rb;
            if (bs != lengths.block || rb != lengths.row_bytes) try_params(c);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    E->params = s == PRAND_OK ? best : keep;
    if (s != PRAND_OK) return s;
    if (seclen_mrg_lfsr) *seclen_mrg_lfsr = best.seclen_mrg_lfsr;
    if (seclen_gm) *seclen_gm = best.seclen_gm;
    if (block) *block = best.block;
    if (row_bytes) *row_bytes = best.row_bytes;
    if (best_ms) *best_ms = best_t;
    const char *path = getenv("PRAND_TUNE_CACHE");
    if (path) {
        FILE *f = fopen(path, "w");
        if (f) {
            fprintf(f, "{\"seclen_mrg_lfsr\": %u, \"seclen_gm\": %u, \"block\": %u, \"row_bytes\": %u, \"ms\": %.4f}\n",
                    best.seclen_mrg_lfsr, best.seclen_gm, best.block, best.row_bytes, best_t);
            fclose(f);
        }
    }
    return PRAND_OK;
}

prand_status_t prand_batch_set_params(uint32_t seclen_mrg_lfsr, uint32_t seclen_gm, uint32_t block, uint32_t row_bytes)
{
    if (seclen_mrg_lfsr == 0 || seclen_gm == 0 || seclen_mrg_lfsr % 4 || seclen_gm % 4 || (block != 64 && block != 128) ||
        (row_bytes != 128 && row_bytes != 256))
        return PRAND_ERR_ARG;
    Engine *E;
    prand_status_t s = engine_get(&E);
    if (s != PRAND_OK) return s;
    E->params.seclen_mrg_lfsr = seclen_mrg_lfsr;
    E->params.seclen_gm = seclen_gm;
    E->params.block = block;
    E->params.row_bytes = row_bytes;
    return PRAND_OK;
}

// Per-request plain launches (for comparison with the fused form): for every
// request, the ordinary stream-initialisation launch(es) and generation launch
// on one stream, with no fusion and no persistent scheduling.
prand_status_t prand_batch_run_per_request(const prand_request_t *reqs, size_t n, uint64_t seed, prand_stream_t stream)
{
    prand_status_t s = validate_requests(reqs, n);
    if (s != PRAND_OK || n == 0) return s;
    cudaStream_t st = (cudaStream_t)stream;
    BatchCtx ctx;
    DevTables *T;
    if ((s = batch_ctx(seed, st, &ctx, &T)) != PRAND_OK) return s;
    size_t maxb = 0;
    for (int g = 0; g < PRAND_NUM_GENERATORS; ++g) maxb = std::max(maxb, state_bytes_per_stream(g));
    void *scratch = nullptr;
    if (n && !dev_alloc(&scratch, 2 * maxb * n)) return PRAND_ERR_NOMEM;
    for (size_t i = 0; i < n && s == PRAND_OK; ++i) {
        const prand_request_t &r = reqs[i];
        if (!r.length) continue;
        void *a = (char *)scratch + 2 * maxb * i, *b = (char *)a + maxb;
        StreamRange R;
        R.stride = R.count = 1;
        uint32_t idx = kMtN;
        if (r.gen == PRAND_MT19937) {
            mt_window_init_kernel<<<1, 32, 0, st>>>((const uint32_t *)ctx.base[r.gen], ctx.mt_win, r.stream,
                                                    (uint32_t *)a);
            s = launch_check();
            if (s == PRAND_OK) s = mt_gen(a, 1, &idx, r.dev_out, r.dtype, r.length, st);
        } else if (is_gm(r.gen)) {
            Variant V;
            variant_params(r.gen, 0, &V);
            s = gm_init(r.gen, T, ctx.base[r.gen], a, r.stream, 1, V, st);
            if (s == PRAND_OK) s = gm_gen(r.gen, T, a, b, R, r.dev_out, r.dtype, r.length, st);
        } else {
            Variant V;
            variant_params(r.gen, 0, &V);
            s = mrg_lfsr_init(r.gen, T, ctx.base[r.gen], a, r.stream, 1, V, st);
            if (s == PRAND_OK) s = mrg_lfsr_gen(r.gen, T, a, b, R, r.dev_out, r.dtype, r.length, st);
        }
    }
    // scratch is freed in stream order (the runtime defers it until the work is done)
    cudaStreamSynchronize(st);
    if (scratch) cudaFree(scratch);
    return s;
}

}  // extern "C"
