// Host SIMD generation of MT19937, LFSR113 and MRG32K3A (the analogue of the
// paper's SSE realisations, Sec. 2 and Table 6): the same outputs as the GPU
// fills, computed on the host's vector units with no GPU involved.
//
// Written with the compiler's generic vector types (16-byte vectors of four
// 32-bit or two 64-bit lanes), so one source becomes SSE2 code on x86-64 and
// NEON code on AArch64; no intrinsics, no inline assembly.
//   MT19937: one stream at a time, the twist four words per vector (Sec. 5.4;
//     a word's partners are the next word and the word 397 ahead, so four
//     consecutive new words never depend on each other), tempering likewise.
//   LFSR113: four streams per vector, one vector per component (Sec. 5.3), so
//     every lane shifts by the same amounts; 4 x 4 blocks of outputs are
//     transposed so each stream's row is stored four outputs at a time.
//   MRG32K3A: two streams per vector of doubles, four vectors in flight
//     (Sec. 5.2).  Each product of
//     a multiplier (< 2^21) and a residue (< 2^32) is exact in a double
//     (< 2^53); the quotient by m is rounded to the nearest integer with the
//     2^52 + 2^51 addition trick, which leaves the remainder in (-m, m), and
//     one conditional add of m makes it canonical.
// Streams are spread over host threads in contiguous ranges.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <type_traits>
#include <vector>

#include "prand.h"
#include "prand_device.h"

namespace {

typedef uint32_t v4u __attribute__((vector_size(16)));
typedef int32_t v4i __attribute__((vector_size(16)));
typedef double v2d __attribute__((vector_size(16)));
typedef uint64_t v2u __attribute__((vector_size(16)));
typedef int64_t v2l __attribute__((vector_size(16)));

inline v4u load4(const uint32_t *p)
{
    v4u v;
    memcpy(&v, p, sizeof v);
    return v;
}
inline void store4(uint32_t *p, v4u v) { memcpy(p, &v, sizeof v); }

// ------------------------------------------------------------ output maps
// The float maps of prand_device.h: f32 = (u >> 8) 2^-24, f64 = u 2^-32,
// MRG32K3A f64 = z RN(1 / (m1 + 1)).
template <typename OutT, bool MRG>
inline OutT conv(uint32_t u);
template <>
inline uint32_t conv<uint32_t, false>(uint32_t u) { return u; }
template <>
inline uint32_t conv<uint32_t, true>(uint32_t u) { return u; }
template <>
inline float conv<float, false>(uint32_t u) { return prand_u32_to_f32(u); }
template <>
inline float conv<float, true>(uint32_t u) { return prand_u32_to_f32(u); }
template <>
inline double conv<double, false>(uint32_t u) { return prand_u32_to_f64(u); }
template <>
inline double conv<double, true>(uint32_t u) { return prand_mrg32k3a_to_f64(u); }

// ------------------------------------------------------------ MT19937
constexpr int kN = 624, kM = 397;

inline v4u mt_recur4(v4u a, v4u b, v4u p)
{
    const v4u y = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
    const v4u mag = (v4u)(-(v4i)(y & 1u)) & 0x9908B0DFu;
    return p ^ (y >> 1) ^ mag;
}

inline uint32_t mt_recur1(uint32_t a, uint32_t b, uint32_t p)
{
    const uint32_t y = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
    return p ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
}

// The whole block in place: new words 0..226 read old words k + 397; words
// 227..623 read new words k - 227 (already written); word 623 reads new word 0.
inline void mt_twist(uint32_t *mt)
{
    int k = 0;
    for (; k + 4 <= kN - kM; k += 4)  // 0..223: all partners old
        store4(mt + k, mt_recur4(load4(mt + k), load4(mt + k + 1), load4(mt + k + kM)));
    for (; k < kN - kM; ++k) mt[k] = mt_recur1(mt[k], mt[k + 1], mt[k + kM]);  // 224..226
    for (; k + 4 <= kN - 1; k += 4)  // 227..622: partners k - 227 are new, k + 1 old
        store4(mt + k, mt_recur4(load4(mt + k), load4(mt + k + 1), load4(mt + k + kM - kN)));
    for (; k < kN - 1; ++k) mt[k] = mt_recur1(mt[k], mt[k + 1], mt[k + kM - kN]);
    mt[kN - 1] = mt_recur1(mt[kN - 1], mt[0], mt[kM - 1]);
}

inline v4u temper4(v4u y)
{
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

template <typename OutT>
void mt_stream(prand_mt19937_state *s, OutT *o, uint64_t n)
{
    uint64_t i = 0;
    while (i < n) {
        if (s->idx >= (uint32_t)kN) {
            mt_twist(s->mt);
            s->idx = 0;
        }
        uint32_t idx = s->idx;
        const uint64_t take = std::min<uint64_t>(n - i, kN - idx);
        uint64_t t = 0;
        for (; t + 4 <= take; t += 4) {
            const v4u v = temper4(load4(s->mt + idx + t));
            for (int e = 0; e < 4; ++e) o[i + t + e] = conv<OutT, false>(v[e]);
        }
        for (; t < take; ++t) {
            const v4u v = temper4((v4u){ s->mt[idx + t], 0, 0, 0 });
            o[i + t] = conv<OutT, false>(v[0]);
        }
        s->idx = idx + (uint32_t)take;
        i += take;
    }
}

// ------------------------------------------------------------ LFSR113
// Component (P, Q, S): (31,6,18), (29,2,2), (28,13,7), (25,3,13).
template <int P, int Q, int S>
inline v4u taus4(v4u z)
{
    constexpr uint32_t mask = 0xFFFFFFFFu << (32 - P);
    return ((z & mask) << S) ^ (((z << Q) ^ z) >> (P - S));
}

// Four streams at once; z[c] holds component c of the four streams.
template <typename OutT>
void lfsr_quad(prand_lfsr113_state *st, OutT *out, uint64_t n, uint64_t row)
{
    v4u z[4];
    for (int c = 0; c < 4; ++c) z[c] = (v4u){ st[0].z[c], st[1].z[c], st[2].z[c], st[3].z[c] };
    uint64_t i = 0;
    for (; i + 4 <= n; i += 4) {
        v4u w[4];
        for (int t = 0; t < 4; ++t) {
            z[0] = taus4<31, 6, 18>(z[0]);
            z[1] = taus4<29, 2, 2>(z[1]);
            z[2] = taus4<28, 13, 7>(z[2]);
            z[3] = taus4<25, 3, 13>(z[3]);
            w[t] = z[0] ^ z[1] ^ z[2] ^ z[3];  // output t of the four streams
        }
        // transpose: stream s's outputs i..i+3 are lane s of w[0..3]
        const v4u a = __builtin_shuffle(w[0], w[1], (v4u){ 0, 4, 1, 5 });
        const v4u b = __builtin_shuffle(w[0], w[1], (v4u){ 2, 6, 3, 7 });
        const v4u c = __builtin_shuffle(w[2], w[3], (v4u){ 0, 4, 1, 5 });
        const v4u d = __builtin_shuffle(w[2], w[3], (v4u){ 2, 6, 3, 7 });
        const v4u r[4] = { __builtin_shuffle(a, c, (v4u){ 0, 1, 4, 5 }), __builtin_shuffle(a, c, (v4u){ 2, 3, 6, 7 }),
                           __builtin_shuffle(b, d, (v4u){ 0, 1, 4, 5 }), __builtin_shuffle(b, d, (v4u){ 2, 3, 6, 7 }) };
        for (int s = 0; s < 4; ++s) {
            OutT *q = out + s * row + i;
            if constexpr (std::is_same<OutT, uint32_t>::value) {  // one 16-byte store
                memcpy(q, &r[s], 16);
            } else {
                for (int e = 0; e < 4; ++e) q[e] = conv<OutT, false>(r[s][e]);
            }
        }
    }
    for (; i < n; ++i) {
        z[0] = taus4<31, 6, 18>(z[0]);
        z[1] = taus4<29, 2, 2>(z[1]);
        z[2] = taus4<28, 13, 7>(z[2]);
        z[3] = taus4<25, 3, 13>(z[3]);
        const v4u w = z[0] ^ z[1] ^ z[2] ^ z[3];
        for (int s = 0; s < 4; ++s) out[s * row + i] = conv<OutT, false>(w[s]);
    }
    for (int s = 0; s < 4; ++s)
        for (int c = 0; c < 4; ++c) st[s].z[c] = z[c][s];
}

// ------------------------------------------------------------ MRG32K3A
constexpr double kM1 = 4294967087.0, kM2 = 4294944443.0;
constexpr double kRound = 6755399441055744.0;  // 2^52 + 2^51: x + kRound - kRound = nearest integer to x

// (a x - b y) mod m for exact integers in doubles: the quotient by m rounded
// to nearest leaves the remainder in (-m, m); one conditional add of m.
inline v2d mod_lin(v2d a_x, v2d b_y, double m, double inv_m)
{
    const v2d p = a_x - b_y;                     // exact: |p| < 2^53
    v2d q = p * inv_m + kRound;
    q = q - kRound;                              // nearest integer to p / m (within one of it)
    v2d r = p - q * m;                           // exact
    const v2l neg = r < 0.0;
    return r + (v2d)((v2l)(v2d){ m, m } & neg);  // add m where r < 0
}

// the low 32 bits of a nonnegative integer below 2^32 held in a double
inline uint32_t u32_of(double x)
{
    return (uint32_t)(int64_t)x;
}

// 2K streams at once (K vectors of two, independent chains for the pipeline);
// x[c][k], y[c][k] hold component c (0: newest) of streams 2k and 2k + 1.
template <typename OutT, int K>
void mrg_group(prand_mrg32k3a_state *st, OutT *out, uint64_t n, uint64_t row)
{
    v2d x[3][K], y[3][K];
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < K; ++k) {
            x[c][k] = (v2d){ (double)st[2 * k].x[c], (double)st[2 * k + 1].x[c] };
            y[c][k] = (v2d){ (double)st[2 * k].y[c], (double)st[2 * k + 1].y[c] };
        }
    const double i1 = 1.0 / kM1, i2 = 1.0 / kM2;
    for (uint64_t i = 0; i < n; ++i) {
        for (int k = 0; k < K; ++k) {
            // x_{n+1} = 1403580 x_{n-1} - 810728 x_{n-2} (mod m1); y_{n+1} = 527612 y_n - 1370589 y_{n-2} (mod m2)
            const v2d xn = mod_lin(1403580.0 * x[1][k], 810728.0 * x[2][k], kM1, i1);
            const v2d yn = mod_lin(527612.0 * y[0][k], 1370589.0 * y[2][k], kM2, i2);
            x[2][k] = x[1][k]; x[1][k] = x[0][k]; x[0][k] = xn;
            y[2][k] = y[1][k]; y[1][k] = y[0][k]; y[0][k] = yn;
            // z = (x - y) mod m1, 0 -> m1: z in [1, m1]
            v2d z = xn - yn;
            const v2l le = z <= 0.0;
            z = z + (v2d)((v2l)(v2d){ kM1, kM1 } & le);
            out[(2 * k) * row + i] = conv<OutT, true>(u32_of(z[0]));
            out[(2 * k + 1) * row + i] = conv<OutT, true>(u32_of(z[1]));
        }
    }
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < 2; ++l) {
            prand_mrg32k3a_state &t = st[2 * k + l];
            t.x[0] = u32_of(x[0][k][l]); t.x[1] = u32_of(x[1][k][l]); t.x[2] = u32_of(x[2][k][l]);
            t.y[0] = u32_of(y[0][k][l]); t.y[1] = u32_of(y[1][k][l]); t.y[2] = u32_of(y[2][k][l]);
        }
}

// ------------------------------------------------------------ dispatch
template <typename OutT>
void run_range(int gen, void *states, uint64_t j0, uint64_t j1, OutT *out, uint64_t n)
{
    if (gen == PRAND_MT19937) {
        prand_mt19937_state *s = (prand_mt19937_state *)states;
        for (uint64_t j = j0; j < j1; ++j) mt_stream<OutT>(s + j, out + j * n, n);
    } else if (gen == PRAND_LFSR113) {
        prand_lfsr113_state *s = (prand_lfsr113_state *)states;
        uint64_t j = j0;
        for (; j + 4 <= j1; j += 4) lfsr_quad<OutT>(s + j, out + j * n, n, n);
        for (; j < j1; ++j)
            for (uint64_t i = 0; i < n; ++i) out[j * n + i] = conv<OutT, false>(prand_lfsr113_next_u32(s + j));
    } else {
        prand_mrg32k3a_state *s = (prand_mrg32k3a_state *)states;
        uint64_t j = j0;
        for (; j + 8 <= j1; j += 8) mrg_group<OutT, 4>(s + j, out + j * n, n, n);
        for (; j + 2 <= j1; j += 2) mrg_group<OutT, 1>(s + j, out + j * n, n, n);
        for (; j < j1; ++j)
            for (uint64_t i = 0; i < n; ++i) out[j * n + i] = conv<OutT, true>(prand_mrg32k3a_next_u32(s + j));
    }
}

template <typename OutT>
void run(int gen, void *states, uint64_t ns, OutT *out, uint64_t n, int threads)
{
    // ranges in multiples of 8 streams, so each thread keeps whole vector groups
    const uint64_t units = (ns + 7) / 8;
    const uint64_t t = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)threads, units));
    if (t == 1) {
        run_range<OutT>(gen, states, 0, ns, out, n);
        return;
    }
    std::vector<std::thread> pool;
    for (uint64_t k = 0; k < t; ++k) {
        const uint64_t a = std::min(ns, units * k / t * 8), b = std::min(ns, units * (k + 1) / t * 8);
        if (a < b) pool.emplace_back(run_range<OutT>, gen, states, a, b, out, n);
    }
    for (auto &th : pool) th.join();
}

}  // namespace

extern "C" prand_status_t prand_host_generate(prand_gen_t gen, int32_t dtype, void *host_states, uint64_t n_streams,
                                              void *host_out, uint64_t n_per_stream, int32_t n_threads)
{
    if (gen != PRAND_MT19937 && gen != PRAND_LFSR113 && gen != PRAND_MRG32K3A) return PRAND_ERR_ARG;
    if (dtype != PRAND_DTYPE_U32 && dtype != PRAND_DTYPE_F32 && dtype != PRAND_DTYPE_F64) return PRAND_ERR_ARG;
    if (n_threads < 0) return PRAND_ERR_ARG;
    if (n_streams == 0 || n_per_stream == 0) return PRAND_OK;
    if (!host_states || !host_out) return PRAND_ERR_ARG;
    const size_t esz = dtype == PRAND_DTYPE_F64 ? 8 : 4;
    if ((uintptr_t)host_out % esz || (uintptr_t)host_states % 4) return PRAND_ERR_ALIGN;
    uint64_t total, bytes;
    if (__builtin_mul_overflow(n_streams, n_per_stream, &total) || __builtin_mul_overflow(total, (uint64_t)esz, &bytes))
        return PRAND_ERR_ARG;
    int threads = n_threads;
    if (threads == 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    // MT19937 states must hold a valid in-block index
    if (gen == PRAND_MT19937) {
        const prand_mt19937_state *s = (const prand_mt19937_state *)host_states;
        for (uint64_t j = 0; j < n_streams; ++j)
            if (s[j].idx > (uint32_t)kN) return PRAND_ERR_STATE;
    }
    if (dtype == PRAND_DTYPE_U32) run<uint32_t>(gen, host_states, n_streams, (uint32_t *)host_out, n_per_stream, threads);
    else if (dtype == PRAND_DTYPE_F32) run<float>(gen, host_states, n_streams, (float *)host_out, n_per_stream, threads);
    else run<double>(gen, host_states, n_streams, (double *)host_out, n_per_stream, threads);
    return PRAND_OK;
}
