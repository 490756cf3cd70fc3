// Request server with continuous batching over the batched persistent kernel.
//
// A request is (generator, stream index, length, element type).  It returns the
// next `length` outputs of that stream: the server keeps every stream it has
// served resident on the device (a state slot), so a later request on the same
// stream continues where the previous one stopped; a stream seen for the first
// time starts from the seeded base advanced by k * L (block splitting, Table 4).
//
// A worker thread admits pending requests in arrival order while output memory
// (a fixed arena) and batch capacity allow, plans their tiles and launches
// them as one batch on one of several CUDA streams, so batches admitted while
// others run overlap on the device.  Requests on a stream that has work in
// flight wait for it (per-stream order).  Each slot is double-buffered: tiles
// read the current half and the request's last tile writes the other, which
// becomes current when the batch completes.  When a generator's slots run out,
// the least recently used idle stream's state moves to host memory and comes
// back on its next request.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <set>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>
#include <algorithm>

#include "batch.cuh"

namespace prand {
namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t esz(int dtype) { return dtype == PRAND_DTYPE_F64 ? 8 : 4; }

// Output arena over [0, cap) in 256-byte units: best fit among the free blocks, found through a size-ordered
// index (O(log n) per allocation however fragmented the arena is), and
// neighbouring free blocks merged on release through the offset-ordered map.
struct Arena {
    std::map<uint64_t, uint64_t> free_;         // offset -> bytes
    std::set<std::pair<uint64_t, uint64_t>> by_size;  // (bytes, offset) of the same blocks
    uint64_t used = 0, top = 0;
    explicit Arena(uint64_t cap = 0)
    {
        if (cap) add(0, cap);
    }
    void add(uint64_t off, uint64_t bytes)
    {
        free_[off] = bytes;
        by_size.emplace(bytes, off);
    }
    void drop(std::map<uint64_t, uint64_t>::iterator it)
    {
        by_size.erase({ it->second, it->first });
        free_.erase(it);
    }
    bool alloc(uint64_t bytes, uint64_t *off)
    {
        bytes = (bytes + 255) & ~255ull;
        auto fit = by_size.lower_bound({ bytes, 0 });
        if (fit == by_size.end()) return false;
        const uint64_t boff = fit->second, bsize = fit->first;
        drop(free_.find(boff));
        if (bsize > bytes) add(boff + bytes, bsize - bytes);
        *off = boff;
        used += bytes;
        top = std::max(top, boff + bytes);
        return true;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        bytes = (bytes + 255) & ~255ull;
        used -= bytes;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {  // merge with the block after
            bytes += nx->second;
            auto after = std::next(nx);
            drop(nx);
            nx = after;
        }
        if (nx != free_.begin()) {  // and with the block before
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                off = pv->first;
                bytes += pv->second;
                drop(pv);
            }
        }
        add(off, bytes);
    }
};

struct Key {
    int gen;
    uint64_t stream;
    bool operator==(const Key &o) const { return gen == o.gen && stream == o.stream; }
};
struct KeyHash {
    size_t operator()(const Key &k) const { return std::hash<uint64_t>()(k.stream * 0x9E3779B97F4A7C15ull + (uint64_t)k.gen); }
};

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct SReq {
    int gen = 0, dtype = 0;
    uint64_t stream = 0, len = 0, off = 0, bytes = 0;
    double t_arr = 0, t_done = 0;
    int state = kPending;
};

struct Resident {
    uint32_t slot = 0;  // slot pair index s: halves 2s and 2s + 1
    uint8_t cur = 0;    // current half
    bool busy = false;  // a request on this stream is in flight
    std::list<uint64_t>::iterator lru;
};

constexpr int kFlights = 32;
constexpr int kMtFlights = 16;  // at most this many flights carry MT19937 batches
// Fixed per-flight capacities, allocated once: growing a buffer in the loop
// would free the old one, and cudaFree / cudaFreeHost wait for the whole
// device, i.e. for every batch in flight.
constexpr size_t kFlightReqs = 2048;    // requests per batch
constexpr size_t kFlightTiles = 32768;  // tiles per batch
constexpr uint32_t kMaxTilesPerRequest = 64;

struct FlightReq {
    uint64_t id;
    Key key;
    uint8_t new_cur;  // the slot half that becomes current when the request is done
    bool done;
};

struct Flight {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr, ev0 = nullptr;  // end and start of the batch on the device
    BatchTile *h_tiles = nullptr, *d_tiles = nullptr;  // kFlightTiles each
    uint32_t *counter = nullptr;
    uint32_t *h_left = nullptr, *d_left = nullptr;  // tiles per request (staging, device countdown)
    volatile uint32_t *h_done = nullptr;            // completed request indices + 1, in completion order (mapped host memory)
    size_t cursor = 0;                              // next h_done entry to read
    std::vector<FlightReq> reqs;
    std::vector<std::vector<uint32_t>> restored;    // host copies of restored states, kept until the batch ends
    size_t ndone = 0;
    int lane = 0;
    bool busy = false;
};

}  // namespace
}  // namespace prand

using namespace prand;

struct prand_server_s {
    int device = -1;
    uint64_t seed = 0;
    BatchCtx ctx;
    BatchParams P;
    char *out_base = nullptr;
    uint64_t out_cap = 0;
    Arena arena;
    void *slot_arena[PRAND_NUM_GENERATORS] = {};
    uint32_t slot_cap = 0;
    std::vector<uint32_t> free_slots[PRAND_NUM_GENERATORS];
    std::unordered_map<Key, Resident, KeyHash> res;
    std::list<uint64_t> lru[PRAND_NUM_GENERATORS];  // stream indices, most recent at the back
    std::unordered_map<Key, std::vector<uint32_t>, KeyHash> spilled;
    // two admission lanes: MT19937 requests (their jump chains take tens of ms)
    // and the rest, so fast batches never wait on a jump chain
    std::deque<uint64_t> pending[2];
    std::unordered_map<uint64_t, SReq> reqs;
    uint64_t next_id = 1;
    uint32_t max_batch_reqs[2] = { 512, 64 };
    Flight fl[kFlights];
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    prand_status_t error = PRAND_OK;
    prand_server_stats_t stats = {};
    std::vector<uint64_t> done_q;  // completed request ids not yet collected
    cudaStream_t aux = nullptr;    // spills (waits only for its own copies)
};

namespace {

// A free slot pair for gen, evicting the least recently used idle stream to
// host memory if needed.  Called with the server lock held.
bool take_slot(prand_server_s *S, int gen, uint32_t *slot)
{
    if (!S->free_slots[gen].empty()) {
        *slot = S->free_slots[gen].back();
        S->free_slots[gen].pop_back();
        return true;
    }
    const size_t words = slot_words(gen);
    for (auto it = S->lru[gen].begin(); it != S->lru[gen].end(); ++it) {
        Key k{ gen, *it };
        auto r = S->res.find(k);
        if (r == S->res.end() || r->second.busy) continue;
        // the stream is idle, so its state was written by a batch whose flag
        // has been seen; the copy runs on its own stream and does not wait for
        // the batches in flight
        std::vector<uint32_t> host(words);
        const uint32_t *src = (const uint32_t *)S->slot_arena[gen] + (2ull * r->second.slot + r->second.cur) * words;
        if (cudaMemcpyAsync(host.data(), src, words * 4, cudaMemcpyDeviceToHost, S->aux) != cudaSuccess ||
            cudaStreamSynchronize(S->aux) != cudaSuccess)
            return false;
        S->spilled[k] = std::move(host);
        *slot = r->second.slot;
        S->lru[gen].erase(r->second.lru);
        S->res.erase(r);
        S->stats.spills++;
        return true;
    }
    return false;
}

void finish_request(prand_server_s *S, FlightReq &q, double t)
{
    q.done = true;
    auto it = S->reqs.find(q.id);
    if (it != S->reqs.end()) {
        it->second.state = kDone;
        it->second.t_done = t;
        S->done_q.push_back(q.id);
        S->stats.completed++;
        S->stats.samples += it->second.len;
    }
    auto r = S->res.find(q.key);
    if (r != S->res.end()) { r->second.cur = q.new_cur; r->second.busy = false; }
}

// Requests complete one by one (the device raises each request's flag when
// its last tile is done), so a request does not wait for slower batch-mates;
// a batch's flight is reused once its event has completed.
void complete_flights(prand_server_s *S)
{
    for (Flight &F : S->fl) {
        if (!F.busy) continue;
        const double t = now_s();
        // new entries of the device's completion list (a slot may be filled out
        // of order; reading stops at the first one not yet written)
        while (F.cursor < F.reqs.size()) {
            const uint32_t v = F.h_done[F.cursor];
            if (v == 0 || v > F.reqs.size()) break;
            FlightReq &q = F.reqs[v - 1];
            if (!q.done) { finish_request(S, q, t); ++F.ndone; }
            ++F.cursor;
        }
        cudaError_t e = cudaEventQuery(F.ev);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) S->error = PRAND_ERR_CUDA;
        float ms = 0;
        if (e == cudaSuccess && cudaEventElapsedTime(&ms, F.ev0, F.ev) == cudaSuccess) S->stats.gpu_busy_s += 1e-3 * ms;
        for (FlightReq &q : F.reqs)
            if (!q.done) finish_request(S, q, t);
        F.reqs.clear();
        F.restored.clear();
        F.ndone = 0;
        F.busy = false;
    }
}

// Plan and launch one batch on flight F from pending lane `lane`.  Lock held.
bool launch_one(prand_server_s *S, Flight &F, int lane)
{
    std::deque<uint64_t> &Q = S->pending[lane];
    const size_t cap = std::min<size_t>(S->max_batch_reqs[lane], kFlightReqs);
    std::vector<BatchTile> tiles;
    std::vector<uint64_t> keep;  // skipped requests, returned to the front of the queue in order
    size_t taken = 0, scanned = 0;
    // Scan the queue in arrival order and stop at the first request that does
    // not fit (output memory) or when the batch is full, so the host work per
    // batch does not grow with the queue; requests on a busy stream are
    // skipped (per-stream order) and keep their place.
    while (!Q.empty() && taken < cap && scanned < 4 * cap) {
        const uint64_t id = Q.front();
        SReq &r = S->reqs[id];
        ++scanned;
        prand_request_t pr;
        pr.gen = r.gen;
        pr.dtype = r.dtype;
        pr.stream = r.stream;
        pr.length = r.len;
        pr.dev_out = nullptr;
        if (tiles.size() + plan_tile_count(pr, S->P, kMaxTilesPerRequest) > kFlightTiles) break;  // batch full
        Key k{ r.gen, r.stream };
        auto ri = S->res.find(k);
        if (ri != S->res.end() && ri->second.busy) {  // per-stream order
            Q.pop_front();
            keep.push_back(id);
            continue;
        }
        // (a later request on a stream taken in this batch finds it busy above)
        uint64_t off;
        if (!S->arena.alloc(r.bytes, &off)) break;  // the oldest waiting request must go first
        Q.pop_front();
        r.off = off;
        int32_t slot = -1, wslot;
        bool from_slot;
        if (ri != S->res.end()) {
            Resident &R = ri->second;
            slot = (int32_t)(2 * R.slot + R.cur);
            wslot = (int32_t)(2 * R.slot + (R.cur ^ 1));
            from_slot = true;
            R.busy = true;
            S->lru[r.gen].erase(R.lru);
            R.lru = S->lru[r.gen].insert(S->lru[r.gen].end(), r.stream);
            F.reqs.push_back({ id, k, (uint8_t)(R.cur ^ 1), false });
            S->stats.hits++;
        } else {
            uint32_t s;
            if (!take_slot(S, r.gen, &s)) { S->arena.release(off, r.bytes); keep.push_back(id); continue; }  // all slots busy
            Resident R;
            R.slot = s;
            R.cur = 0;
            R.busy = true;
            R.lru = S->lru[r.gen].insert(S->lru[r.gen].end(), r.stream);
            auto sp = S->spilled.find(k);
            if (sp != S->spilled.end()) {
                // restore an evicted state into half 0 (ordered before the batch on this stream)
                const size_t words = slot_words(r.gen);
                uint32_t *dst = (uint32_t *)S->slot_arena[r.gen] + (2ull * s) * words;
                // ordered before the batch on the flight's stream; the host copy
                // stays alive until the batch has finished
                F.restored.push_back(std::move(sp->second));
                if (cudaMemcpyAsync(dst, F.restored.back().data(), words * 4, cudaMemcpyHostToDevice, F.st) != cudaSuccess)
                    S->error = PRAND_ERR_CUDA;
                S->spilled.erase(sp);
                slot = (int32_t)(2 * s);
                from_slot = true;
                S->stats.restores++;
            } else {
                from_slot = false;
                S->stats.misses++;
            }
            wslot = (int32_t)(2 * s + 1);
            S->res[k] = R;
            F.reqs.push_back({ id, k, (uint8_t)1, false });
        }
        pr.dev_out = S->out_base + off;
        const size_t before = tiles.size();
        plan_request(pr, slot, wslot, from_slot, S->P, tiles, kMaxTilesPerRequest);
        for (size_t i = before; i < tiles.size(); ++i) tiles[i].req = (uint32_t)(F.reqs.size() - 1);
        r.state = kRunning;
        ++taken;
    }
    for (size_t i = keep.size(); i-- > 0;) Q.push_front(keep[i]);
    if (F.reqs.empty()) return false;
    const size_t nr = F.reqs.size();
    if (S->error == PRAND_OK) {
        memset(F.h_left, 0, nr * 4);
        for (const BatchTile &t : tiles) F.h_left[t.req]++;
        for (size_t i = 0; i < nr; ++i) F.h_done[i] = 0;
        F.cursor = 0;
    }
    // the fast lane's tiles are alike: no sort, but the thread-per-stream GM/GQ
    // tiles go first (their kernel build runs before the rest's)
    if (lane == 1) order_tiles(tiles);
    else std::stable_partition(tiles.begin(), tiles.end(), [](const BatchTile &t) { return wide_tile_gen(t.gen); });
    const size_t n = tiles.size();
    if (S->error == PRAND_OK) {
        memcpy(F.h_tiles, tiles.data(), n * sizeof(BatchTile));
        BatchCtx ctx = S->ctx;
        ctx.tiles_left = F.d_left;
        ctx.done_list = F.h_done;
        ctx.done_count = F.counter + 4;  // its own 16-byte slot of the flight's counter block
        if (cudaEventRecord(F.ev0, F.st) != cudaSuccess ||
            cudaMemsetAsync(F.counter + 4, 0, sizeof(uint32_t), F.st) != cudaSuccess ||
            cudaMemcpyAsync(F.d_tiles, F.h_tiles, n * sizeof(BatchTile), cudaMemcpyHostToDevice, F.st) != cudaSuccess ||
            cudaMemcpyAsync(F.d_left, F.h_left, nr * 4, cudaMemcpyHostToDevice, F.st) != cudaSuccess ||
            launch_batch(F.d_tiles, (uint32_t)n, count_mt_tiles(tiles),
                         count_wide_tiles(tiles, count_mt_tiles(tiles)), F.counter, ctx, F.st) != PRAND_OK ||
            cudaEventRecord(F.ev, F.st) != cudaSuccess)
            S->error = PRAND_ERR_CUDA;
    }
    F.ndone = 0;
    F.busy = true;
    S->stats.batches++;
    S->stats.tiles += n;
    return true;
}

// Queue one request (the server lock held).
prand_status_t submit_locked(prand_server_s *S, int32_t gen, uint64_t stream, uint64_t length, int32_t dtype,
                             uint64_t *id)
{
    if (gen < 0 || gen >= PRAND_NUM_GENERATORS || dtype < 0 || dtype > 2 || length == 0) return PRAND_ERR_ARG;
    uint64_t bytes;
    if (__builtin_mul_overflow(length, (uint64_t)esz(dtype), &bytes) || ((bytes + 255) & ~255ull) > S->out_cap)
        return PRAND_ERR_ARG;  // can never fit the output arena
    if (S->error != PRAND_OK) return S->error;
    SReq r;
    r.gen = gen;
    r.dtype = dtype;
    r.stream = stream;
    r.len = length;
    r.bytes = bytes;
    r.t_arr = now_s();
    *id = S->next_id++;
    S->reqs[*id] = r;
    S->pending[gen == PRAND_MT19937 ? 1 : 0].push_back(*id);
    return PRAND_OK;
}

void worker_loop(prand_server_s *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        complete_flights(S);
        bool launched = false;
        int mt_busy = 0;
        for (Flight &F : S->fl) mt_busy += F.busy && F.lane == 1;
        const double tb = now_s();
        for (int lane = 0; lane < 2 && !launched; ++lane) {
            if (S->pending[lane].empty()) continue;
            if (lane == 1 && mt_busy >= kMtFlights) continue;  // the rest of the flights stay with the fast lane
            for (Flight &F : S->fl)
                if (!F.busy) { F.lane = lane; launched = launch_one(S, F, lane); break; }
        }
        if (launched) S->stats.worker_busy_s += now_s() - tb;
        if (launched) continue;
        bool any_busy = false;
        for (Flight &F : S->fl) any_busy = any_busy || F.busy;
        // wake on a submission, or poll the in-flight batches every 20 us
        S->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 2000));
    }
}

}  // namespace

extern "C" {

prand_status_t prand_server_create(prand_server_t *out, uint64_t seed, uint64_t output_bytes, uint32_t slots_per_generator)
{
    if (!out || output_bytes < 256 || slots_per_generator == 0) return PRAND_ERR_ARG;
    *out = nullptr;
    prand_server_t S = new (std::nothrow) prand_server_s;
    if (!S) return PRAND_ERR_NOMEM;
    auto fail = [&](prand_status_t e) {
        for (Flight &F : S->fl) {
            if (F.ev) cudaEventDestroy(F.ev);
            if (F.ev0) cudaEventDestroy(F.ev0);
            if (F.st) cudaStreamDestroy(F.st);
            if (F.counter) cudaFree(F.counter);
            if (F.d_tiles) cudaFree(F.d_tiles);
            if (F.h_tiles) cudaFreeHost(F.h_tiles);
            if (F.d_left) cudaFree(F.d_left);
            if (F.h_left) cudaFreeHost(F.h_left);
            if (F.h_done) cudaFreeHost((void *)F.h_done);
        }
        if (S->aux) cudaStreamDestroy(S->aux);
        for (int g = 0; g < PRAND_NUM_GENERATORS; ++g) if (S->slot_arena[g]) cudaFree(S->slot_arena[g]);
        if (S->out_base) cudaFree(S->out_base);
        delete S;
        return e;
    };
    if (cudaGetDevice(&S->device) != cudaSuccess) return fail(PRAND_ERR_CUDA);
    S->seed = seed;
    prand_status_t s = batch_ctx(seed, 0, &S->ctx, nullptr);
    if (s != PRAND_OK) return fail(s);
    // The tuned launch shape of this GPU, with the server's own section
    // lengths: requests are short and latency counts, so 2048 outputs per lane
    // for MRG32K3A / LFSR113 sections whatever the batch tuner chose for
    // throughput (8192: p50 4.5 ms against 1.0 ms at the serving load).
    S->P = batch_params();
    S->P.seclen_mrg_lfsr = 2048;
    S->P.seclen_gm = 8192;
    S->out_cap = output_bytes & ~255ull;
    if (!dev_alloc(&S->out_base, S->out_cap)) { S->out_base = nullptr; return fail(PRAND_ERR_NOMEM); }
    S->arena = Arena(S->out_cap);
    S->slot_cap = slots_per_generator;
    // Every resident stream holds a slot, so the map of resident streams never
    // outgrows the slots: sized for them now, it is never rehashed under the
    // lock while batches wait (a rehash of a few hundred thousand streams took
    // tens of milliseconds in the middle of a serving run).  The same for the
    // requests in the server at once and the streams moved to host memory.
    try {
        S->res.reserve((size_t)slots_per_generator * PRAND_NUM_GENERATORS);
        S->reqs.reserve(2 * kFlights * kFlightReqs);
        S->spilled.reserve((size_t)slots_per_generator * PRAND_NUM_GENERATORS);
    } catch (const std::bad_alloc &) {
        return fail(PRAND_ERR_NOMEM);
    }
    for (int g = 0; g < PRAND_NUM_GENERATORS; ++g) {
        const size_t bytes = 2ull * slots_per_generator * slot_words(g) * 4;
        if (!dev_alloc(&S->slot_arena[g], bytes)) { S->slot_arena[g] = nullptr; return fail(PRAND_ERR_NOMEM); }
        S->ctx.slots[g] = S->slot_arena[g];
        S->free_slots[g].reserve(slots_per_generator);
        for (uint32_t i = slots_per_generator; i-- > 0;) S->free_slots[g].push_back(i);
    }
    for (Flight &F : S->fl) {
        if (cudaStreamCreateWithFlags(&F.st, cudaStreamNonBlocking) != cudaSuccess) return fail(PRAND_ERR_CUDA);
        if (cudaEventCreate(&F.ev) != cudaSuccess || cudaEventCreate(&F.ev0) != cudaSuccess) return fail(PRAND_ERR_CUDA);
        if (!dev_alloc(&F.counter, 64)) return fail(PRAND_ERR_NOMEM);
        void *hd = nullptr;
        if (!host_alloc(&F.h_tiles, kFlightTiles * sizeof(BatchTile)) ||
            !dev_alloc(&F.d_tiles, kFlightTiles * sizeof(BatchTile)) ||
            !host_alloc(&F.h_left, kFlightReqs * 4) ||
            !dev_alloc(&F.d_left, kFlightReqs * 4) ||
            !host_alloc(&hd, kFlightReqs * 4, cudaHostAllocMapped))
            return fail(PRAND_ERR_NOMEM);
        F.h_done = (volatile uint32_t *)hd;
    }
    if (cudaStreamCreateWithFlags(&S->aux, cudaStreamNonBlocking) != cudaSuccess) return fail(PRAND_ERR_CUDA);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return PRAND_OK;
}

prand_status_t prand_server_submit(prand_server_t S, int32_t gen, uint64_t stream, uint64_t length, int32_t dtype,
                                   uint64_t *id)
{
    if (!S || !id) return PRAND_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    prand_status_t s = submit_locked(S, gen, stream, length, dtype, id);
    if (s == PRAND_OK) S->cv.notify_one();
    return s;
}

prand_status_t prand_server_query(prand_server_t S, uint64_t id, int32_t *done, void **dev_out, double *latency_s)
{
    if (!S) return PRAND_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return PRAND_ERR_ARG;
    const SReq &r = it->second;
    if (done) *done = r.state == kDone;
    if (dev_out) *dev_out = r.state == kDone ? (void *)(S->out_base + r.off) : nullptr;
    if (latency_s) *latency_s = r.state == kDone ? r.t_done - r.t_arr : -1.0;
    return S->error;
}

prand_status_t prand_server_read(prand_server_t S, uint64_t id, void *host_dst, uint64_t bytes)
{
    if (!S || !host_dst) return PRAND_ERR_ARG;
    const char *src;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || it->second.state != kDone) return PRAND_ERR_STATE;
        if (bytes > it->second.bytes) return PRAND_ERR_ARG;
        src = S->out_base + it->second.off;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->device) cudaSetDevice(S->device);
    const cudaError_t e = cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost);
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    return e == cudaSuccess ? PRAND_OK : PRAND_ERR_CUDA;
}

prand_status_t prand_server_release(prand_server_t S, uint64_t id)
{
    if (!S) return PRAND_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second.state != kDone) return PRAND_ERR_STATE;
    S->arena.release(it->second.off, it->second.bytes);
    S->reqs.erase(it);
    S->cv.notify_one();
    return PRAND_OK;
}

prand_status_t prand_server_stats(prand_server_t S, prand_server_stats_t *out)
{
    if (!S || !out) return PRAND_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->pending = S->pending[0].size() + S->pending[1].size();
    out->arena_used_bytes = S->arena.used;
    out->arena_free_blocks = S->arena.free_.size();
    out->arena_top_bytes = S->arena.top;
    out->flights_busy = 0;
    for (const Flight &F : S->fl) out->flights_busy += F.busy;
    return S->error;
}

prand_status_t prand_server_destroy(prand_server_t S)
{
    if (!S) return PRAND_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_one();
    }
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (Flight &F : S->fl) {
        if (F.st) cudaStreamSynchronize(F.st);
        if (F.ev) cudaEventDestroy(F.ev);
        if (F.ev0) cudaEventDestroy(F.ev0);
        if (F.st) cudaStreamDestroy(F.st);
        if (F.counter) cudaFree(F.counter);
        if (F.d_tiles) cudaFree(F.d_tiles);
        if (F.h_tiles) cudaFreeHost(F.h_tiles);
        if (F.d_left) cudaFree(F.d_left);
        if (F.h_left) cudaFreeHost(F.h_left);
        if (F.h_done) cudaFreeHost((void *)F.h_done);
    }
    if (S->aux) cudaStreamDestroy(S->aux);
    for (int g = 0; g < PRAND_NUM_GENERATORS; ++g) if (S->slot_arena[g]) cudaFree(S->slot_arena[g]);
    if (S->out_base) cudaFree(S->out_base);
    delete S;
    return PRAND_OK;
}

prand_status_t prand_server_completed(prand_server_t S, uint64_t *ids, size_t cap, size_t *n)
{
    if (!S || !n || (!ids && cap)) return PRAND_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    const size_t k = std::min(cap, S->done_q.size());
    if (k) {
        memcpy(ids, S->done_q.data(), k * sizeof(uint64_t));
        S->done_q.erase(S->done_q.begin(), S->done_q.begin() + (ptrdiff_t)k);
    }
    *n = k;
    return S->error;
}

// Open-loop load driver: submits request i at arrival_s[i] seconds after the
// call starts (a native thread keeps the schedule), releases each output as
// soon as it completes, and returns every request's latency (arrival ->
// completion).  For measuring the server; the outputs are not kept.
prand_status_t prand_server_replay(prand_server_t S, const prand_request_t *reqs, const double *arrival_s, size_t n,
                                   double *latency_s, double *wall_s)
{
    if (!S || (!reqs && n) || (!arrival_s && n) || (!latency_s && n)) return PRAND_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->done_q.clear();
    }
    std::unordered_map<uint64_t, size_t> index;
    index.reserve(2 * n);
    std::vector<std::pair<uint64_t, double>> fin;
    const double t0 = now_s();
    size_t next = 0, done = 0;
    prand_status_t err = PRAND_OK;
    while (done < n && err == PRAND_OK) {
        const double t = now_s() - t0;
        // submit every request that has arrived, under one lock
        if (next < n && arrival_s[next] <= t) {
            std::lock_guard<std::mutex> lk(S->mu);
            while (next < n && arrival_s[next] <= t) {
                const prand_request_t &r = reqs[next];
                uint64_t id;
                err = submit_locked(S, r.gen, r.stream, r.length, r.dtype, &id);
                if (err != PRAND_OK) break;
                index[id] = next;
                ++next;
            }
            S->cv.notify_one();
        }
        // collect and release every completed request under one lock
        fin.clear();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->error != PRAND_OK) err = S->error;
            for (uint64_t id : S->done_q) {
                auto it = S->reqs.find(id);
                if (it == S->reqs.end()) continue;
                fin.emplace_back(id, it->second.t_done - it->second.t_arr);
                S->arena.release(it->second.off, it->second.bytes);
                S->reqs.erase(it);
            }
            S->done_q.clear();
            if (!fin.empty()) S->cv.notify_one();
        }
        const size_t k = fin.size();
        for (const auto &f : fin) {
            auto it = index.find(f.first);
            if (it != index.end()) { latency_s[it->second] = f.second; index.erase(it); ++done; }
        }
        if (k == 0 && next < n && arrival_s[next] > now_s() - t0 + 50e-6)
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        else if (k == 0 && next >= n)
            std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (wall_s) *wall_s = now_s() - t0;
    return err;
}

}  // extern "C"
