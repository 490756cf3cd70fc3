// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "prand.h"

namespace prand {

// ---------------------------------------------------------------------------
// Allocation.  A refused cudaMalloc / cudaHostAlloc also leaves its error in
// the runtime's per-thread last-error slot, where the next launch check
// (cudaGetLastError) would find it and report a launch that succeeded as a
// CUDA failure.  These wrappers clear it, so a refused allocation is reported
// once, as PRAND_ERR_NOMEM by the caller, and later calls are unaffected.
// ---------------------------------------------------------------------------
template <typename T>
inline bool dev_alloc(T **p, size_t bytes)
{
    if (cudaMalloc((void **)p, bytes) == cudaSuccess) return true;
    *p = nullptr;
    (void)cudaGetLastError();
    return false;
}

template <typename T>
inline bool host_alloc(T **p, size_t bytes, unsigned flags = cudaHostAllocDefault)
{
    if (cudaHostAlloc((void **)p, bytes, flags) == cudaSuccess) return true;
    *p = nullptr;
    (void)cudaGetLastError();
    return false;
}

// ---------------------------------------------------------------------------
// Generator constants, restated from the paper.
// ---------------------------------------------------------------------------

// MT19937 (Matsumoto & Nishimura 1998; Sec. 5.4).
constexpr int kMtN = 624;
constexpr int kMtM = 397;
constexpr int kMtDeg = 19937;          // state dimension over GF(2)
constexpr int kMtPolyWords = 624;      // 32-bit words per jump polynomial (19968 bits)
constexpr int kMtPolyCount = 512;      // stored x^(2^b) mod phi, b = 0..511 (Sec. 5.4)
constexpr int kMtStreamShift = 432;    // L = 2^432 >= 1e130 (Table 4)
constexpr int kMtWinBits = 8;          // stream jumps by digits of 8 bits (bytes) of the stream index
constexpr int kMtWinDigits = 1 << kMtWinBits;
constexpr int kMtWinPositions = 64 / kMtWinBits;  // digit positions of a 64-bit stream index

// MRG32K3A (Sec. 5.2).
constexpr uint32_t kM1 = 4294967087u;  // 2^32 - 209
constexpr uint32_t kM2 = 4294944443u;  // 2^32 - 22853
constexpr int kMrgStreamShift = 127;   // L = 2^127 >= 1e38 (Table 4)

// LFSR113 (Sec. 5.3): (p, q, s) per component.
constexpr int kLfsrStreamShift = 34;   // L = 2^34 >= 1e10 (Table 4)

// Jump tables hold M^(2^b) for b < kJumpBits (offsets up to 2^256).
constexpr int kJumpBits = 256;

// GM / GQ ensembles (Sec. 5.1, Table 2).  All arithmetic is done on z = x / 2^t
// modulo the prime p (for GM55 and GQ58.x, g = 2^t p and k, q are even, so the
// states used here are multiples of 2^t and x = 2^t z follows the same map mod p).
enum PrimeKind { P19 = 0, P29 = 1, P31 = 2, P51 = 3, P61 = 4 };

struct GmParams {
    uint64_t k, q, p;  // recurrence z' = k z - q z_prev (mod p)
    int t;             // g = 2^t p
    int v;             // output bits per point
    int s;             // points per output word
    int lanes;         // lanes per stream: 32 (one lane per point) or 1 (one thread per stream)
    PrimeKind kind;
    uint64_t L;        // block length (Table 4 maximal length)
    uint64_t nmax;     // number of sequences (Table 4)
};

inline bool is_gm(int gen) { return gen >= PRAND_GM19 && gen <= PRAND_GQ58_4; }

// SM count of the current device, from the runtime (1 if the query fails: the
// next CUDA call then reports the error).
inline int device_sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 1;
    return sms;
}
const GmParams &gm_params(int gen);

// Block length L as a 64-bit value for GM/GQ and the Table 4 capacity per generator.
uint64_t table4_nmax(int gen);

// A stream-initialisation variant of Table 4 (0: init_sequence or
// init_short_sequence, 1: init_medium_sequence, 2: init_long_sequence): its
// number of sequences, block length L and, for GM/GQ, the spacing D = N_max L
// of the ensemble's points, the last two as 128-bit little-endian values.
// MRG32K3A and MT19937 have variant 0 only, with L = 2^127 and 2^432 (not
// representable here; their kernels use the shift).  False if Table 4 does not
// list the variant.
struct Variant {
    uint64_t nmax = 0;
    uint64_t L[2] = { 0, 0 };
    uint64_t D[2] = { 0, 0 };
};
bool variant_params(int gen, int v, Variant *out);

// ---------------------------------------------------------------------------
// Per-device jump tables.
// ---------------------------------------------------------------------------
struct DevTables {
    int device = -1;
    uint32_t *mrg = nullptr;      // [kJumpBits][18]: A^(2^b) mod m1 (9 words), B^(2^b) mod m2 (9 words)
    uint32_t *lfsr = nullptr;     // [4][kJumpBits][32]: column images of T_c^(2^b)
    uint64_t *gm[8] = {};         // per GM/GQ generator: [kJumpBits][4] = M^(2^b) mod p
    uint32_t *mt = nullptr;       // [kMtPolyCount][kMtPolyWords]: x^(2^b) mod phi
    uint32_t *mt_win = nullptr;   // [kMtWinPositions][kMtWinDigits][kMtPolyWords]: x^(d 2^(432 + 8 i)) mod phi
    bool ready_basic = false;
    bool ready_mt = false;
    bool ready_mt_win = false;
};

// Returns the tables of the current device, building what `gen` needs.
prand_status_t get_tables(int gen, DevTables **out);

// Host side of the MT19937 jump: characteristic polynomial (Berlekamp-Massey)
// and the squaring chain x^(2^b) mod phi, b < count; each polynomial as 624
// little-endian 32-bit words.  Computed once per process.
const uint32_t *mt_host_pow2_polys();
// x^(d 2^(432 + 8 i)) mod phi for the 8 byte positions i of a stream index and
// digits d = 1..255 ([i][d][624 words], d = 0 unused): a stream jump is one
// polynomial application per nonzero byte (about 8 for a random 64-bit index,
// against about 15 with hex digits).  Computed once per process, on all host
// cores.
const uint32_t *mt_host_window_polys();
// The device copy of that table for the current device (built on first use).
prand_status_t get_mt_window(DevTables *T);

// ---------------------------------------------------------------------------
// Handles.
// ---------------------------------------------------------------------------
struct prand_handle_impl;

// Counting launches (all kernels go through launch_check()).
extern std::atomic<uint64_t> g_launches;
prand_status_t launch_check();  // cudaGetLastError after a launch; counts it

// Offsets as 256-bit little-endian numbers.
struct U256 { uint64_t w[4]; };

// The streams one fill covers: streams j0 .. j0 + count - 1 of state arrays
// laid out for `stride` streams.  Sections: nsec == 0 lets the family choose
// (nsec and seclen are written back); otherwise the given pair is used, so the
// fills of several ranges in one call split their streams alike and keep their
// next states in the same buffer (in place when nsec == 1, the spare otherwise).
struct StreamRange {
    uint64_t stride = 0, j0 = 0, count = 0;
    uint32_t nsec = 0;
    uint64_t seclen = 0;
};

// Sections per stream for a launch of `units` work items (threads or lane
// groups, one per stream) with nper outputs each, when `cap` items are
// resident at once: the count in [1, max_s] whose grid best fills whole waves,
// discounted for the fixed work each section starts with (its jump, state
// load and store: about 128 outputs' worth).  Candidates: 1..64, multiples of one wave's worth, max_s.
inline uint32_t pick_nsec(uint64_t units, uint64_t cap, uint64_t max_s, uint64_t nper)
{
    if (cap == 0 || units == 0 || nper == 0) return 1;
    if (max_s < 1) max_s = 1;
    if (max_s > 65535) max_s = 65535;
    auto score = [&](uint64_t s) {
        const uint64_t n = units * s, waves = (n + cap - 1) / cap;
        return ((double)n / (double)(waves * cap)) / (1.0 + 128.0 * (double)s / (double)nper);
    };
    uint64_t best = 1;
    double best_score = score(1);
    auto consider = [&](uint64_t s) {
        if (s < 1 || s > max_s) return;
        const double v = score(s);
        if (v > best_score + 1e-9) { best_score = v; best = s; }
    };
    for (uint64_t s = 2; s <= 64; ++s) consider(s);
    const uint64_t wave = (cap + units - 1) / units;  // sections per stream for one full wave
    for (uint64_t k = 1; k <= 8; ++k) consider(k * wave);
    consider(max_s);
    return (uint32_t)best;
}

// Family entry points (gen_mrg_lfsr.cu, gm_dispatch.cpp, gen_mt.cu), all
// asynchronous on `st`.  The *_gen functions fill `out` (stream-major, R.count
// rows of nper) from the streams of R and leave their next states in place or,
// when R.nsec > 1, in the spare buffer (the caller swaps the two afterwards).
prand_status_t mrg_build_table(uint32_t *tab, cudaStream_t st);
prand_status_t lfsr_build_table(uint32_t *tab, cudaStream_t st);
prand_status_t gm_build_table(int gen, uint64_t *tab, cudaStream_t st);
prand_status_t mrg_lfsr_seed(int gen, uint64_t seed, void *d_base, cudaStream_t st);
prand_status_t mrg_lfsr_init(int gen, const DevTables *T, const void *d_base, void *d_state, uint64_t first, uint64_t n,
                             const Variant &V, cudaStream_t st);
prand_status_t mrg_lfsr_skip(int gen, const DevTables *T, void *d_state, uint64_t n, const U256 &off, cudaStream_t st);
prand_status_t mrg_lfsr_gen(int gen, const DevTables *T, void *d_state, void *d_spare, StreamRange &R, void *out,
                            int dtype, uint64_t nper, cudaStream_t st);
prand_status_t gm_seed(int gen, const DevTables *T, uint64_t seed, const Variant &V, void *d_base, cudaStream_t st);
prand_status_t gm_init(int gen, const DevTables *T, const void *d_base, void *d_state, uint64_t first, uint64_t n,
                       const Variant &V, cudaStream_t st);
prand_status_t gm_skip(int gen, const DevTables *T, void *d_state, uint64_t n, const U256 &off, cudaStream_t st);
prand_status_t gm_gen(int gen, const DevTables *T, void *d_state, void *d_spare, StreamRange &R, void *out, int dtype,
                      uint64_t nper, cudaStream_t st);
prand_status_t mt_seed(uint64_t seed, void *d_base, cudaStream_t st);
// Streams first..first+n-1, stream k = base advanced by k * 2^shift (the
// Table 4 block length 2^432 by default; shift + 63 < kMtPolyCount).
prand_status_t mt_init(const DevTables *T, const void *d_base, void *d_state, uint64_t first, uint64_t n, cudaStream_t st,
                       int shift = kMtStreamShift);
prand_status_t mt_skip(const DevTables *T, void *d_state, uint64_t n, uint32_t *idx, const U256 &off, cudaStream_t st);
prand_status_t mt_skip512(const DevTables *T, void *d_state, uint64_t n, uint32_t *idx, const uint64_t off[8],
                          cudaStream_t st);
// MT19937 keeps its state as 624-word blocks per stream (a range is a pointer
// offset); *idx, the position inside the block shared by all streams, advances.
prand_status_t mt_gen(void *d_state, uint64_t nstreams, uint32_t *idx, void *out, int dtype, uint64_t nper, cudaStream_t st);

// States in the prand_device.h layout (states.cu): bytes per stream (0 for an
// unknown generator), and the copies out of / into a handle's state arrays
// (the import of MT19937 states checks that all share one block index and
// waits for `st`).
uint64_t device_state_bytes(int gen);
prand_status_t export_states_dev(int gen, const void *d_state, uint64_t n, uint32_t mt_idx, void *out, cudaStream_t st);
prand_status_t import_states_dev(int gen, const void *in, uint64_t n, void *d_state, uint32_t *mt_idx, cudaStream_t st);

// Family-specific device work, all asynchronous on `st` unless noted.
// Base state of one "stream" in the family's device layout.
prand_status_t seed_base(int gen, uint64_t seed, void *d_base, cudaStream_t st);
// State bytes per stream in the family's device layout.
size_t state_bytes_per_stream(int gen);
// streams j = 0..n-1 := base advanced by (first + j) * L
prand_status_t init_streams_dev(int gen, const DevTables *T, const void *d_base, void *d_state,
                                uint64_t first, uint64_t n, cudaStream_t st);
// all streams += off
prand_status_t skipahead_dev(int gen, const DevTables *T, void *d_state, uint64_t n, uint32_t *mt_idx,
                             const U256 &off, cudaStream_t st);
// generate
prand_status_t generate_dev(int gen, const DevTables *T, void *d_state, uint64_t nstreams, uint32_t *mt_idx,
                            void *out, int dtype, uint64_t nper, cudaStream_t st);

}  // namespace prand
