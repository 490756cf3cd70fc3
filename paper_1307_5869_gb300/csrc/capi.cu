// The prand_* C ABI: handle management, per-device jump tables, argument
// checking, and dispatch to the generator families.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "prand_internal.h"

namespace prand {

std::atomic<uint64_t> g_launches{ 0 };

prand_status_t launch_check()
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError() == cudaSuccess ? PRAND_OK : PRAND_ERR_CUDA;
}

size_t state_bytes_per_stream(int gen)
{
    if (gen == PRAND_MT19937) return kMtN * sizeof(uint32_t);
    if (gen == PRAND_MRG32K3A) return 6 * sizeof(uint32_t);
    if (gen == PRAND_LFSR113) return 4 * sizeof(uint32_t);
    return 2 * (size_t)gm_params(gen).s * sizeof(uint64_t);
}

bool variant_params(int gen, int v, Variant *out)
{
    // Table 4: (number of sequences, maximal length) of each initialisation
    // function; the block length is the printed maximal length for GM/GQ and
    // the power of two above it for LFSR113 (2^34, 2^80).
    using u128 = unsigned __int128;
    const u128 e7 = 10000000ull, e9 = 1000000000ull, e10 = 10000000000ull;
    uint64_t nm = 0;
    u128 L = 0;
    switch (gen) {
    case PRAND_GM19: if (v == 0) { nm = 1000; L = 6000000; } break;
    case PRAND_GM29: case PRAND_GQ58_1: case PRAND_GQ58_3: case PRAND_GQ58_4: {
        const uint64_t f = gen == PRAND_GQ58_3 ? 2 : gen == PRAND_GQ58_4 ? 3 : 1;
        if (v == 0) { nm = f * 100000000ull; L = 8 * e7; }
        else if (v == 1) { nm = f * 1000000ull; L = 8 * e9; }
        else if (v == 2) { nm = f * 10000ull; L = 800 * e9; }
        break;
    }
    case PRAND_GM31:
        if (v == 0) { nm = 1000000000ull; L = 8 * e7; }
        else if (v == 1) { nm = 10000000ull; L = 8 * e9; }
        else if (v == 2) { nm = 100000ull; L = 800 * e9; }
        break;
    case PRAND_GM55:
        if (v == 0) { nm = 1000000000000000000ull; L = e10; }
        else if (v == 2) { nm = 4000000000ull; L = e10 * e10; }
        break;
    case PRAND_GM61:
        if (v == 0) { nm = 18000000000000000000ull; L = e10; }
        else if (v == 2) { nm = 4000000000ull; L = 300000 * e10 * e10; }
        break;
    case PRAND_LFSR113:
        if (v == 0) { nm = 3800000000000000000ull; L = (u128)1 << 34; }
        else if (v == 2) { nm = 4000000000ull; L = (u128)1 << 80; }
        break;
    case PRAND_MRG32K3A:
        if (v == 0) { nm = 10000000000000000000ull; L = (u128)1 << kMrgStreamShift; }
        break;
    case PRAND_MT19937:
        if (v == 0) nm = 10000000000000000000ull;  // L = 2^432 (above 128 bits): applied as a shift
        break;
    default: break;
    }
    if (!nm) return false;
    out->nmax = nm;
    out->L[0] = (uint64_t)L;
    out->L[1] = (uint64_t)(L >> 64);
    const u128 D = L * nm;  // below 2^117 for every GM/GQ variant
    out->D[0] = is_gm(gen) ? (uint64_t)D : 0;
    out->D[1] = is_gm(gen) ? (uint64_t)(D >> 64) : 0;
    return true;
}

// Handle layouts: a Table 4 variant (0, 1, 2), or streams spaced 2^s apart
// (kSpacedTag + s; the skip-ahead layout of Table 3).  The GM/GQ base of a
// spaced layout is the default variant's ensemble.
constexpr int32_t kSpacedTag = 0x10000;
constexpr int kMaxSpacing = 127, kMaxSpacingMt = kMtPolyCount - 64;

static bool layout_params(int gen, int32_t layout, Variant *V, int *mt_shift)
{
    *mt_shift = kMtStreamShift;
    if (layout < kSpacedTag) return variant_params(gen, layout, V);
    const int sp = layout - kSpacedTag;
    if (sp > (gen == PRAND_MT19937 ? kMaxSpacingMt : kMaxSpacing) || !variant_params(gen, 0, V)) return false;
    V->L[0] = sp < 64 ? 1ull << sp : 0;
    V->L[1] = sp >= 64 ? 1ull << (sp - 64) : 0;
    V->nmax = UINT64_MAX;  // a chosen spacing has no Table 4 capacity
    *mt_shift = sp;
    return true;
}

uint64_t table4_nmax(int gen)
{
    if (gen == PRAND_MT19937 || gen == PRAND_MRG32K3A) return 10000000000000000000ull;  // 1e19
    if (gen == PRAND_LFSR113) return 3800000000000000000ull;                            // 3.8e18
    return gm_params(gen).nmax;
}

// ------------------------------------------------------------------ tables
namespace {
constexpr int kMaxDevices = 64;
DevTables g_tables[kMaxDevices];
std::mutex g_tables_mu;
}  // namespace

prand_status_t get_mt_window(DevTables *T)
{
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if (T->ready_mt_win) return PRAND_OK;
    const uint32_t *host = mt_host_window_polys();
    if (!host) return PRAND_ERR_STATE;
    const size_t bytes = (size_t)kMtWinPositions * kMtWinDigits * kMtPolyWords * sizeof(uint32_t);
    if (!dev_alloc(&T->mt_win, bytes)) return PRAND_ERR_NOMEM;
    if (cudaMemcpy(T->mt_win, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return PRAND_ERR_CUDA;
    T->ready_mt_win = true;
    return PRAND_OK;
}

prand_status_t get_tables(int gen, DevTables **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PRAND_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_tables_mu);
    DevTables &T = g_tables[dev];
    T.device = dev;
    if (!T.ready_basic) {
        size_t mrg_b = (size_t)kJumpBits * 18 * sizeof(uint32_t);
        size_t lfsr_b = (size_t)4 * kJumpBits * 32 * sizeof(uint32_t);
        size_t gm_b = (size_t)kJumpBits * 4 * sizeof(uint64_t);
        if (!dev_alloc(&T.mrg, mrg_b)) return PRAND_ERR_NOMEM;
        if (!dev_alloc(&T.lfsr, lfsr_b)) return PRAND_ERR_NOMEM;
        for (int g = 0; g < 8; ++g)
            if (!dev_alloc(&T.gm[g], gm_b)) return PRAND_ERR_NOMEM;
        prand_status_t s = mrg_build_table(T.mrg, 0);
        if (s == PRAND_OK) s = lfsr_build_table(T.lfsr, 0);
        for (int g = 0; g < 8 && s == PRAND_OK; ++g) s = gm_build_table(PRAND_GM19 + g, T.gm[g], 0);
        if (s == PRAND_OK && cudaDeviceSynchronize() != cudaSuccess) s = PRAND_ERR_CUDA;
        if (s != PRAND_OK) return s;
        T.ready_basic = true;
    }
    if (gen == PRAND_MT19937 && !T.ready_mt) {
        const uint32_t *host = mt_host_pow2_polys();
        if (!host) return PRAND_ERR_STATE;
        size_t bytes = (size_t)kMtPolyCount * kMtPolyWords * sizeof(uint32_t);
        if (!dev_alloc(&T.mt, bytes)) return PRAND_ERR_NOMEM;
        if (cudaMemcpy(T.mt, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return PRAND_ERR_CUDA;
        T.ready_mt = true;
    }
    *out = &T;
    return PRAND_OK;
}

}  // namespace prand

using namespace prand;

struct prand_handle_s {
    int gen = 0;
    uint64_t seed = 0;
    int device = 0;
    DevTables *T = nullptr;
    void *d_base = nullptr;
    void *d_state = nullptr;
    void *d_spare = nullptr;
    uint64_t first = 0, n = 0;
    uint64_t position = 0;
    int variant = 0;       // Table 4 variant of the streams
    int base_variant = 0;  // variant the base state was seeded for (GM/GQ ensembles differ)
    uint32_t mt_idx = kMtN;
    cudaStream_t last_stream = 0;
    // host fills: two device staging buffers, a copy stream and its events
    void *stage[2] = {};
    uint64_t stage_bytes = 0;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_gen[2] = {}, ev_copy[2] = {};
};

namespace {

constexpr uint32_t kBlobMagic = 0x444E5250u;  // "PRND"
constexpr uint32_t kBlobVersion = 2;  // 2: the stream variant follows the state sizes

struct BlobHeader {
    uint32_t magic, version;
    int32_t gen;
    uint32_t mt_idx;
    uint64_t seed, first, n, position, state_bytes;
    int32_t variant;
    uint32_t reserved;
};

prand_status_t check_device(prand_handle_t h)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PRAND_ERR_CUDA;
    return dev == h->device ? PRAND_OK : PRAND_ERR_STATE;
}

prand_status_t sync_last(prand_handle_t h)
{
    return cudaStreamSynchronize(h->last_stream) == cudaSuccess ? PRAND_OK : PRAND_ERR_CUDA;
}

void free_states(prand_handle_t h)
{
    if (h->d_state) cudaFree(h->d_state);
    if (h->d_spare) cudaFree(h->d_spare);
    h->d_state = h->d_spare = nullptr;
    h->n = 0;
}

bool mul_overflows(uint64_t a, uint64_t b, uint64_t *r)
{
    return __builtin_mul_overflow(a, b, r);
}

prand_status_t generate_any(prand_handle_t h, void *out, int dtype, uint64_t nper, prand_stream_t stream)
{
    if (!h || !out) return PRAND_ERR_ARG;
    size_t esz = dtype == PRAND_DTYPE_F64 ? 8 : 4;
    if ((uintptr_t)out % esz) return PRAND_ERR_ALIGN;
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    uint64_t total, bytes;
    if (mul_overflows(h->n, nper, &total) || mul_overflows(total, esz, &bytes)) return PRAND_ERR_ARG;
    if (nper == 0) return PRAND_OK;
    cudaStream_t st = (cudaStream_t)stream;
    StreamRange R;
    R.stride = R.count = h->n;
    if (h->gen == PRAND_MT19937) s = mt_gen(h->d_state, h->n, &h->mt_idx, out, dtype, nper, st);
    else if (is_gm(h->gen)) s = gm_gen(h->gen, h->T, h->d_state, h->d_spare, R, out, dtype, nper, st);
    else s = mrg_lfsr_gen(h->gen, h->T, h->d_state, h->d_spare, R, out, dtype, nper, st);
    if (s != PRAND_OK) return s;
    if (R.nsec > 1) { void *t = h->d_state; h->d_state = h->d_spare; h->d_spare = t; }
    h->position += nper;
    h->last_stream = st;
    return PRAND_OK;
}

// Staging for host fills, allocated on first use: 256 MiB per buffer unless
// PRAND_HOST_STAGE_BYTES asks for another size (at least 4 KiB).
constexpr uint64_t kStageBytesDefault = 256ull << 20;

void free_staging(prand_handle_t h)
{
    for (int b = 0; b < 2; ++b) {
        if (h->stage[b]) cudaFree(h->stage[b]);
        if (h->ev_gen[b]) cudaEventDestroy(h->ev_gen[b]);
        if (h->ev_copy[b]) cudaEventDestroy(h->ev_copy[b]);
        h->stage[b] = nullptr;
        h->ev_gen[b] = h->ev_copy[b] = nullptr;
    }
    if (h->copy_st) cudaStreamDestroy(h->copy_st);
    h->copy_st = nullptr;
    h->stage_bytes = 0;
}

prand_status_t ensure_staging(prand_handle_t h)
{
    if (h->stage[0]) return PRAND_OK;
    uint64_t bytes = kStageBytesDefault;
    if (const char *e = getenv("PRAND_HOST_STAGE_BYTES")) {
        const unsigned long long v = strtoull(e, nullptr, 10);
        if (v >= 4096) bytes = (uint64_t)v & ~255ull;
    }
    h->stage_bytes = bytes;
    bool ok = cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = dev_alloc(&h->stage[b], bytes) &&
             cudaEventCreateWithFlags(&h->ev_gen[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->ev_copy[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        free_staging(h);
        return PRAND_ERR_NOMEM;
    }
    return PRAND_OK;
}

// The device address of host_out when the device can write it directly: a
// page-locked host allocation (under unified addressing every page-locked
// allocation is mapped into the device's address space).  nullptr for
// pageable memory, which goes through the staged copies below.
void *mapped_host_address(void *host_out)
{
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, host_out) != cudaSuccess) {
        cudaGetLastError();  // an unknown pointer is not an error of a later launch
        return nullptr;
    }
    return pa.type == cudaMemoryTypeHost ? pa.devicePointer : nullptr;
}

// The host-array fill.  Page-locked host_out: the generation kernels write the
// outputs straight into it over the host link (no staging buffer, no copy
// engine; a compute-bound generator then costs no more than its device fill).
// Pageable host_out: the outputs are generated on the device in blocks of
// (streams x outputs) that fit a staging buffer and copied into host_out, the
// copy of one block overlapping the generation of the next (two buffers, two
// streams).  Output blocks run in order; within one, the stream blocks share
// one section split, so their next states land in the same buffer.  Either
// way the outputs are in host_out when the call returns.
prand_status_t generate_host(prand_handle_t h, void *host_out, int dtype, uint64_t nper, prand_stream_t stream)
{
    if (!h || !host_out) return PRAND_ERR_ARG;
    const size_t esz = dtype == PRAND_DTYPE_F64 ? 8 : 4;
    if ((uintptr_t)host_out % esz) return PRAND_ERR_ALIGN;
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    uint64_t total, bytes;
    if (mul_overflows(h->n, nper, &total) || mul_overflows(total, esz, &bytes)) return PRAND_ERR_ARG;
    if (nper == 0) return PRAND_OK;
    if (void *mapped = mapped_host_address(host_out)) {
        s = generate_any(h, mapped, dtype, nper, stream);
        if (s == PRAND_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) s = PRAND_ERR_CUDA;
        return s;
    }
    if ((s = ensure_staging(h)) != PRAND_OK) return s;
    const uint64_t n = h->n, stage = h->stage_bytes;
    // outputs per block: whole rows when 65536 streams (or all) fit, else
    // shorter rows (multiples of 64 outputs)
    const uint64_t rows = std::min<uint64_t>(n, 65536);
    uint64_t k = nper;
    if (k > stage / (esz * rows)) k = std::max<uint64_t>(64, (stage / (esz * rows)) & ~63ull);
    if (k > nper) k = nper;
    const uint64_t cs = std::max<uint64_t>(1, std::min<uint64_t>(n, stage / (k * esz)));
    cudaStream_t st = (cudaStream_t)stream;
    char *host = (char *)host_out;
    uint64_t c = 0;
    for (uint64_t i0 = 0; i0 < nper && s == PRAND_OK; i0 += k) {
        const uint64_t kk = std::min(k, nper - i0);
        StreamRange proto;
        proto.stride = n;
        const uint32_t idx0 = h->mt_idx;
        uint32_t idx_next = idx0;
        for (uint64_t j0 = 0; j0 < n && s == PRAND_OK; j0 += cs, ++c) {
            const uint64_t cnt = std::min(cs, n - j0);
            const int b = (int)(c & 1);
            if (c >= 2 && cudaStreamWaitEvent(st, h->ev_copy[b], 0) != cudaSuccess) { s = PRAND_ERR_CUDA; break; }
            void *dst = h->stage[b];
            if (h->gen == PRAND_MT19937) {
                uint32_t idx = idx0;
                s = mt_gen((uint32_t *)h->d_state + j0 * kMtN, cnt, &idx, dst, dtype, kk, st);
                idx_next = idx;
            } else {
                StreamRange R = proto;
                R.j0 = j0;
                R.count = cnt;
                if (is_gm(h->gen)) s = gm_gen(h->gen, h->T, h->d_state, h->d_spare, R, dst, dtype, kk, st);
                else s = mrg_lfsr_gen(h->gen, h->T, h->d_state, h->d_spare, R, dst, dtype, kk, st);
                proto.nsec = R.nsec;
                proto.seclen = R.seclen;
            }
            if (s != PRAND_OK) break;
            char *hdst = host + (j0 * nper + i0) * esz;
            if (cudaEventRecord(h->ev_gen[b], st) != cudaSuccess ||
                cudaStreamWaitEvent(h->copy_st, h->ev_gen[b], 0) != cudaSuccess) {
                s = PRAND_ERR_CUDA;
                break;
            }
            // whole rows are one contiguous piece of host_out; partial rows are strided
            const cudaError_t ce =
                kk == nper ? cudaMemcpyAsync(hdst, dst, cnt * kk * esz, cudaMemcpyDeviceToHost, h->copy_st)
                           : cudaMemcpy2DAsync(hdst, nper * esz, dst, kk * esz, kk * esz, cnt, cudaMemcpyDeviceToHost,
                                               h->copy_st);
            if (ce != cudaSuccess || cudaEventRecord(h->ev_copy[b], h->copy_st) != cudaSuccess) s = PRAND_ERR_CUDA;
        }
        if (s != PRAND_OK) break;
        h->mt_idx = idx_next;
        if (proto.nsec > 1) { void *t = h->d_state; h->d_state = h->d_spare; h->d_spare = t; }
        h->position += kk;
    }
    // the copies into host_out are complete (or abandoned) before returning
    if (cudaStreamSynchronize(h->copy_st) != cudaSuccess && s == PRAND_OK) s = PRAND_ERR_CUDA;
    h->last_stream = st;
    return s;
}

}  // namespace

extern "C" {

prand_status_t prand_create(prand_handle_t *out, prand_gen_t gen, uint64_t seed)
{
    if (!out) return PRAND_ERR_ARG;
    *out = nullptr;
    if ((int)gen < 0 || (int)gen >= PRAND_NUM_GENERATORS) return PRAND_ERR_ARG;
    prand_handle_t h = new (std::nothrow) prand_handle_s;
    if (!h) return PRAND_ERR_NOMEM;
    h->gen = (int)gen;
    h->seed = seed;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return PRAND_ERR_CUDA; }
    prand_status_t s = get_tables(h->gen, &h->T);
    if (s != PRAND_OK) { delete h; return s; }
    if (!dev_alloc(&h->d_base, state_bytes_per_stream(h->gen))) { delete h; return PRAND_ERR_NOMEM; }
    Variant V;
    variant_params(h->gen, 0, &V);
    if (h->gen == PRAND_MT19937) s = mt_seed(seed, h->d_base, 0);
    else if (is_gm(h->gen)) s = gm_seed(h->gen, h->T, seed, V, h->d_base, 0);
    else s = mrg_lfsr_seed(h->gen, seed, h->d_base, 0);
    if (s == PRAND_OK && cudaStreamSynchronize(0) != cudaSuccess) s = PRAND_ERR_CUDA;
    if (s != PRAND_OK) { cudaFree(h->d_base); delete h; return s; }
    *out = h;
    return PRAND_OK;
}

static prand_status_t init_layout(prand_handle_t h, int32_t layout, uint64_t first_stream, uint64_t n_streams)
{
    if (!h || n_streams == 0) return PRAND_ERR_ARG;
    Variant V;
    int mt_shift;
    if (!layout_params(h->gen, layout, &V, &mt_shift)) return PRAND_ERR_ARG;
    uint64_t last;
    if (__builtin_add_overflow(first_stream, n_streams - 1, &last)) return PRAND_ERR_ARG;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    if ((s = sync_last(h)) != PRAND_OK) return s;
    const int base_variant = layout < kSpacedTag ? layout : 0;
    if (is_gm(h->gen) && base_variant != h->base_variant) {
        // the GM/GQ ensemble is spaced for its variant: seed the base again
        if ((s = gm_seed(h->gen, h->T, h->seed, V, h->d_base, 0)) != PRAND_OK) return s;
        h->base_variant = base_variant;
    }
    h->variant = layout;
    free_states(h);
    uint64_t bytes;
    if (mul_overflows(n_streams, state_bytes_per_stream(h->gen), &bytes)) return PRAND_ERR_ARG;
    if (!dev_alloc(&h->d_state, bytes)) { h->d_state = nullptr; return PRAND_ERR_NOMEM; }
    if (h->gen != PRAND_MT19937 && !dev_alloc(&h->d_spare, bytes)) {
        h->d_spare = nullptr;
        free_states(h);
        return PRAND_ERR_NOMEM;
    }
    if (h->gen == PRAND_MT19937) s = mt_init(h->T, h->d_base, h->d_state, first_stream, n_streams, 0, mt_shift);
    else if (is_gm(h->gen)) s = gm_init(h->gen, h->T, h->d_base, h->d_state, first_stream, n_streams, V, 0);
    else s = mrg_lfsr_init(h->gen, h->T, h->d_base, h->d_state, first_stream, n_streams, V, 0);
    if (s == PRAND_OK && cudaStreamSynchronize(0) != cudaSuccess) s = PRAND_ERR_CUDA;
    if (s != PRAND_OK) { free_states(h); return s; }
    h->first = first_stream;
    h->n = n_streams;
    h->position = 0;
    h->mt_idx = kMtN;
    h->last_stream = 0;
    // Table 4 capacity: the last stream index must stay below the number of sequences
    if (last >= V.nmax) return PRAND_WARN_STREAM_OVERLAP;
    return PRAND_OK;
}

prand_status_t prand_init_streams_variant(prand_handle_t h, int32_t variant, uint64_t first_stream, uint64_t n_streams)
{
    if (variant < 0 || variant >= kSpacedTag) return PRAND_ERR_ARG;
    return init_layout(h, variant, first_stream, n_streams);
}

prand_status_t prand_init_streams(prand_handle_t h, uint64_t first_stream, uint64_t n_streams)
{
    return init_layout(h, 0, first_stream, n_streams);
}

prand_status_t prand_init_streams_spaced(prand_handle_t h, uint32_t log2_spacing, uint64_t first_stream,
                                         uint64_t n_streams)
{
    if (log2_spacing > (uint32_t)kMaxSpacingMt) return PRAND_ERR_ARG;
    return init_layout(h, kSpacedTag + (int32_t)log2_spacing, first_stream, n_streams);
}

prand_status_t prand_generate_u32(prand_handle_t h, uint32_t *dev_out, uint64_t n_per_stream, prand_stream_t stream)
{
    return generate_any(h, dev_out, PRAND_DTYPE_U32, n_per_stream, stream);
}

prand_status_t prand_generate_f32(prand_handle_t h, float *dev_out, uint64_t n_per_stream, prand_stream_t stream)
{
    return generate_any(h, dev_out, PRAND_DTYPE_F32, n_per_stream, stream);
}

prand_status_t prand_generate_f64(prand_handle_t h, double *dev_out, uint64_t n_per_stream, prand_stream_t stream)
{
    return generate_any(h, dev_out, PRAND_DTYPE_F64, n_per_stream, stream);
}

prand_status_t prand_generate_host_u32(prand_handle_t h, uint32_t *host_out, uint64_t n_per_stream, prand_stream_t stream)
{
    return generate_host(h, host_out, PRAND_DTYPE_U32, n_per_stream, stream);
}

prand_status_t prand_generate_host_f32(prand_handle_t h, float *host_out, uint64_t n_per_stream, prand_stream_t stream)
{
    return generate_host(h, host_out, PRAND_DTYPE_F32, n_per_stream, stream);
}

prand_status_t prand_generate_host_f64(prand_handle_t h, double *host_out, uint64_t n_per_stream, prand_stream_t stream)
{
    return generate_host(h, host_out, PRAND_DTYPE_F64, n_per_stream, stream);
}

prand_status_t prand_mt_jump_polynomial(uint32_t b, uint32_t *host_out)
{
    if (b >= (uint32_t)kMtPolyCount || !host_out) return PRAND_ERR_ARG;
    const uint32_t *polys = mt_host_pow2_polys();
    if (!polys) return PRAND_ERR_STATE;
    memcpy(host_out, polys + (size_t)b * kMtPolyWords, (size_t)kMtPolyWords * sizeof(uint32_t));
    return PRAND_OK;
}

uint64_t prand_device_state_bytes(prand_gen_t gen)
{
    return (gen < 0 || gen >= PRAND_NUM_GENERATORS) ? 0 : device_state_bytes((int)gen);
}

prand_status_t prand_export_states(prand_handle_t h, void *dev_states, prand_stream_t stream)
{
    if (!h || !dev_states) return PRAND_ERR_ARG;
    if ((uintptr_t)dev_states % (is_gm(h->gen) ? 8 : 4)) return PRAND_ERR_ALIGN;
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    s = export_states_dev(h->gen, h->d_state, h->n, h->mt_idx, dev_states, (cudaStream_t)stream);
    if (s == PRAND_OK) h->last_stream = (cudaStream_t)stream;
    return s;
}

prand_status_t prand_import_states(prand_handle_t h, const void *dev_states, prand_stream_t stream)
{
    if (!h || !dev_states) return PRAND_ERR_ARG;
    if ((uintptr_t)dev_states % (is_gm(h->gen) ? 8 : 4)) return PRAND_ERR_ALIGN;
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    s = import_states_dev(h->gen, dev_states, h->n, h->d_state, &h->mt_idx, (cudaStream_t)stream);
    if (s == PRAND_OK) h->last_stream = (cudaStream_t)stream;
    return s;
}

prand_status_t prand_skipahead(prand_handle_t h, const uint64_t offset_le[4])
{
    if (!h || !offset_le) return PRAND_ERR_ARG;
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    if ((s = sync_last(h)) != PRAND_OK) return s;
    U256 off;
    for (int i = 0; i < 4; ++i) off.w[i] = offset_le[i];
    if (!(off.w[0] | off.w[1] | off.w[2] | off.w[3])) return PRAND_OK;
    if (h->gen == PRAND_MT19937) s = mt_skip(h->T, h->d_state, h->n, &h->mt_idx, off, 0);
    else if (is_gm(h->gen)) s = gm_skip(h->gen, h->T, h->d_state, h->n, off, 0);
    else s = mrg_lfsr_skip(h->gen, h->T, h->d_state, h->n, off, 0);
    if (s == PRAND_OK && cudaStreamSynchronize(0) != cudaSuccess) s = PRAND_ERR_CUDA;
    if (s == PRAND_OK) h->position += off.w[0];
    return s;
}

prand_status_t prand_skipahead_pow2(prand_handle_t h, uint64_t a, uint32_t b)
{
    if (!h) return PRAND_ERR_ARG;
    if (a == 0) return PRAND_OK;
    const uint32_t bits = b + (64 - (uint32_t)__builtin_clzll(a));  // bit length of a 2^b
    if (b >= 512 || bits > (h->gen == PRAND_MT19937 ? 512u : 256u)) return PRAND_ERR_ARG;
    uint64_t w[8] = {};
    w[b / 64] = a << (b % 64);
    if (b % 64 && b / 64 + 1 < 8) w[b / 64 + 1] = a >> (64 - b % 64);
    if (h->gen != PRAND_MT19937) return prand_skipahead(h, w);
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    if ((s = sync_last(h)) != PRAND_OK) return s;
    s = mt_skip512(h->T, h->d_state, h->n, &h->mt_idx, w, 0);
    if (s == PRAND_OK && cudaStreamSynchronize(0) != cudaSuccess) s = PRAND_ERR_CUDA;
    if (s == PRAND_OK) h->position += w[0];
    return s;
}

prand_status_t prand_get_state(prand_handle_t h, void *host_buf, size_t *bytes)
{
    if (!h || !bytes) return PRAND_ERR_ARG;
    if (!h->d_state || h->n == 0) return PRAND_ERR_STATE;
    size_t sb = (size_t)h->n * state_bytes_per_stream(h->gen);
    size_t need = sizeof(BlobHeader) + sb;
    if (!host_buf) { *bytes = need; return PRAND_OK; }
    if (*bytes < need) { *bytes = need; return PRAND_ERR_ARG; }
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    if ((s = sync_last(h)) != PRAND_OK) return s;
    BlobHeader hd = { kBlobMagic, kBlobVersion, h->gen, h->mt_idx, h->seed, h->first, h->n, h->position, sb, h->variant, 0 };
    memcpy(host_buf, &hd, sizeof hd);
    if (cudaMemcpy((char *)host_buf + sizeof hd, h->d_state, sb, cudaMemcpyDeviceToHost) != cudaSuccess) return PRAND_ERR_CUDA;
    *bytes = need;
    return PRAND_OK;
}

prand_status_t prand_set_state(prand_handle_t h, const void *host_buf, size_t bytes)
{
    if (!h || !host_buf || bytes < sizeof(BlobHeader)) return PRAND_ERR_ARG;
    BlobHeader hd;
    memcpy(&hd, host_buf, sizeof hd);
    Variant V;
    int mt_shift;
    if (hd.magic != kBlobMagic || hd.version != kBlobVersion || hd.gen != h->gen || hd.n == 0 ||
        !layout_params(h->gen, hd.variant, &V, &mt_shift))
        return PRAND_ERR_STATE;
    uint64_t sb;
    if (mul_overflows(hd.n, state_bytes_per_stream(h->gen), &sb) || sb != hd.state_bytes ||
        bytes != sizeof hd + sb || hd.mt_idx > (uint32_t)kMtN)
        return PRAND_ERR_STATE;
    prand_status_t s = check_device(h);
    if (s != PRAND_OK) return s;
    if ((s = sync_last(h)) != PRAND_OK) return s;
    if (h->n != hd.n) {
        free_states(h);
        if (!dev_alloc(&h->d_state, sb)) { h->d_state = nullptr; return PRAND_ERR_NOMEM; }
        if (h->gen != PRAND_MT19937 && !dev_alloc(&h->d_spare, sb)) {
            h->d_spare = nullptr;
            free_states(h);
            return PRAND_ERR_NOMEM;
        }
    }
    if (cudaMemcpy(h->d_state, (const char *)host_buf + sizeof hd, sb, cudaMemcpyHostToDevice) != cudaSuccess) return PRAND_ERR_CUDA;
    h->first = hd.first;
    h->n = hd.n;
    h->position = hd.position;
    h->mt_idx = hd.mt_idx;
    h->variant = hd.variant;
    return PRAND_OK;
}

prand_status_t prand_query(prand_handle_t h, uint64_t *first_stream, uint64_t *n_streams, uint64_t *position)
{
    if (!h) return PRAND_ERR_ARG;
    if (first_stream) *first_stream = h->first;
    if (n_streams) *n_streams = h->n;
    if (position) *position = h->position;
    return PRAND_OK;
}

prand_status_t prand_destroy(prand_handle_t h)
{
    if (!h) return PRAND_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    cudaStreamSynchronize(h->last_stream);
    free_states(h);
    free_staging(h);
    if (h->d_base) cudaFree(h->d_base);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    delete h;
    return PRAND_OK;
}

const char *prand_status_string(prand_status_t s)
{
    switch (s) {
    case PRAND_OK: return "success";
    case PRAND_ERR_ARG: return "invalid argument";
    case PRAND_ERR_ALIGN: return "output pointer not aligned to its element size";
    case PRAND_ERR_NOMEM: return "out of memory";
    case PRAND_ERR_CUDA: return "CUDA error";
    case PRAND_ERR_STATE: return "invalid handle state or state blob";
    case PRAND_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PRAND_WARN_STREAM_OVERLAP: return "streams beyond the generator's Table 4 capacity may overlap";
    default: return "unknown status";
    }
}

uint64_t prand_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
