// MRG32K3A (Sec. 5.2) and LFSR113 (Sec. 5.3): seeding, jump tables, block
// splitting, skip-ahead and multi-stream generation.
//
// Both generators keep their whole state in registers (6 and 4 words), so one
// thread runs one section of one stream: sections of a stream start at
// multiples of the section length, reached by the exact jump (A^n, B^n mod m;
// GF(2) powers of the LFSR word step), exactly as the paper's array fill
// splits an array into sections (Sec. 6).  State is stored structure-of-arrays
// (word c of stream j at state[c * nstreams + j]) so a warp loads it coalesced.
#include <array>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "mrg_lfsr_dev.cuh"

namespace prand {

// ------------------------------------------------ section jumps of one fill
// The sections of a fill start at s * seclen (s = 1 .. nsec - 1) in every
// stream, so the jump to each section start is the same matrix for all
// streams.  For up to kSecJumps sections these matrices are built once on the
// host and passed as a kernel parameter: a section thread then applies one
// matrix instead of one table entry per set bit of its offset.
constexpr int kSecJumps = 15;
struct NoSecJumps {
    static constexpr int kCount = 0;
};
struct LfsrSecJumps {
    static constexpr int kCount = kSecJumps;
    uint32_t col[kSecJumps][4][32];  // [s - 1][component][bit]: image of bit i under T_c^(s seclen)
};
// MRG32K3A: section s < 16^4 reached by one matrix per nonzero base-16 digit
// d_j of s (A^(d_j 16^j seclen) commute, so their order does not matter): at
// most four 3x3 products however many sections a fill has, so a single stream
// can be split into sections of 64 outputs (one table entry per set bit of the
// offset would cost up to 14 dependent products per section).
struct MrgSecJumps {
    static constexpr int kLevels = 4;
    static constexpr uint32_t kMaxSections = 1u << (4 * kLevels);
    uint32_t m[kLevels][15][18];  // [j][d - 1]: A^(d 16^j seclen) mod m1, B^(...) mod m2, row-major
};

template <typename SJ>
__device__ __forceinline__ void lfsr_jump_section(const uint32_t *tab, const SJ &sj, uint64_t sec, uint64_t start,
                                                  uint32_t z[4])
{
    if constexpr (SJ::kCount > 0) {
        if (sec <= (uint64_t)SJ::kCount) {
            for (int c = 0; c < 4; ++c) z[c] = gf2_apply(sj.col[sec - 1][c], z[c]);
            return;
        }
    }
    for (int b = 0; b < 64; ++b)
        if ((start >> b) & 1u) lfsr_apply_bit(tab, b, z);
}

template <typename SJ>
__device__ __forceinline__ void mrg_jump_section(const uint32_t *tab, const SJ &sj, uint64_t sec, uint64_t start,
                                                 uint32_t x[3], uint32_t y[3])
{
    if constexpr (!std::is_same<SJ, NoSecJumps>::value) {
        if (sec < (uint64_t)SJ::kMaxSections) {
#pragma unroll
            for (int j = 0; j < SJ::kLevels; ++j) {
                const uint32_t d = (uint32_t)(sec >> (4 * j)) & 15u;
                if (d) {
                    mat3_vec<209>(sj.m[j][d - 1], x);
                    mat3_vec<22853>(sj.m[j][d - 1] + 9, y);
                }
            }
            return;
        }
    }
    for (int b = 0; b < 64; ++b)
        if ((start >> b) & 1u) mrg_apply_bit(tab, b, x, y);
}

// =========================================================== MRG32K3A
// tab[b] = (A^(2^b) mod m1, B^(2^b) mod m2), b < kJumpBits.
__global__ void mrg_table_kernel(uint32_t *tab)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t A[9], B[9];
    mrg_step_matrices(A, B);
    for (int b = 0; b < kJumpBits; ++b) {
        for (int i = 0; i < 9; ++i) { tab[18 * b + i] = A[i]; tab[18 * b + 9 + i] = B[i]; }
        mat3_sqr<209>(A);
        mat3_sqr<22853>(B);
    }
}

// Default state: all six words 12345 (the paper does not print it; L'Ecuyer's
// package default).  Seeded: SplitMix64 draws, x mod m1, y mod m2, never all zero.
__global__ void mrg_seed_kernel(uint32_t *base, uint64_t seed)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (seed == PRAND_SEED_DEFAULT) {
        for (int i = 0; i < 6; ++i) base[i] = 12345u;
        return;
    }
    uint64_t sm = seed;
    uint32_t x[3], y[3];
    do { for (int i = 0; i < 3; ++i) x[i] = (uint32_t)(splitmix64_next(sm) % kM1); } while (!(x[0] | x[1] | x[2]));
    do { for (int i = 0; i < 3; ++i) y[i] = (uint32_t)(splitmix64_next(sm) % kM2); } while (!(y[0] | y[1] | y[2]));
    for (int i = 0; i < 3; ++i) { base[i] = x[i]; base[3 + i] = y[i]; }
}

// k * L for a 64-bit k and a 128-bit L: the exact 192-bit product.
__device__ __forceinline__ void mul_64x128(uint64_t k, uint64_t llo, uint64_t lhi, uint64_t e[3])
{
    e[0] = k * llo;
    const uint64_t c0 = __umul64hi(k, llo);
    e[1] = k * lhi + c0;
    e[2] = __umul64hi(k, lhi) + (e[1] < c0 ? 1u : 0u);
}

// Stream j = base advanced by (first + j) * L, L of 128 bits (2^127 in the
// Table 4 layout); the exponent of up to 192 bits is exact.
__global__ void mrg_init_kernel(const uint32_t *tab, const uint32_t *base, uint32_t *state, uint64_t first, uint64_t n,
                                uint64_t llo, uint64_t lhi)
{
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t x[3] = { base[0], base[1], base[2] }, y[3] = { base[3], base[4], base[5] };
    uint64_t e[3];
    mul_64x128(first + j, llo, lhi, e);
    for (int w = 0; w < 3; ++w)
        for (int b = 0; e[w] && b < 64; ++b)
            if ((e[w] >> b) & 1u) mrg_apply_bit(tab, 64 * w + b, x, y);
    for (int i = 0; i < 3; ++i) { state[i * n + j] = x[i]; state[(3 + i) * n + j] = y[i]; }
}

__global__ void mrg_skip_kernel(const uint32_t *tab, uint32_t *state, uint64_t n, U256 off)
{
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t x[3], y[3];
    for (int i = 0; i < 3; ++i) { x[i] = state[i * n + j]; y[i] = state[(3 + i) * n + j]; }
    for (int b = 0; b < kJumpBits; ++b)
        if (u256_bit(off, b)) mrg_apply_bit(tab, b, x, y);
    for (int i = 0; i < 3; ++i) { state[i * n + j] = x[i]; state[(3 + i) * n + j] = y[i]; }
}

// One thread = one section of one stream.  Sections have length seclen (the
// last one may be shorter); the thread of the last section writes the stream's
// next state to sout, a separate buffer when a stream has several sections (so
// no thread reads a state that another thread has already replaced).
template <typename OutT, bool ROWS = false, typename SJ = NoSecJumps>
__global__ void __launch_bounds__(256) mrg_gen_kernel(const uint32_t *__restrict__ tab, const uint32_t *state, uint32_t *sout, uint64_t nstreams,
                                                      uint64_t stride, uint64_t nper, uint32_t nsec, uint64_t seclen,
                                                      OutT *__restrict__ out, int vec, const __grid_constant__ SJ sj)
{
    uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ROWS) {
        // every lane of a warp takes part in the staged stores (256 threads per block)
        __shared__ __align__(16) unsigned char tiles[8][kTileBytes];
        const bool live = tid < nstreams * nsec;
        const uint64_t j = live ? tid % nstreams : 0;
        const uint64_t start = live ? (tid / nstreams) * seclen : 0;
        const uint64_t len = (live && start < nper) ? min(seclen, nper - start) : 0;
        uint32_t x0 = 0, x1 = 0, x2 = 0, y0 = 0, y1 = 0, y2 = 0;
        if (len) {
            x0 = state[j]; x1 = state[stride + j]; x2 = state[2 * stride + j];
            y0 = state[3 * stride + j]; y1 = state[4 * stride + j]; y2 = state[5 * stride + j];
            if (start) {
                uint32_t x[3] = { x0, x1, x2 }, y[3] = { y0, y1, y2 };
                mrg_jump_section(tab, sj, tid / nstreams, start, x, y);
                x0 = x[0]; x1 = x[1]; x2 = x[2]; y0 = y[0]; y1 = y[1]; y2 = y[2];
            }
        }
        fill_rows<OutT>([&]() { return mrg_next(x0, x1, x2, y0, y1, y2); },
                        [](uint32_t u) { return Cvt<OutT, true>::f(u); }, out + j * nper + start, len,
                        tiles[threadIdx.x >> 5], threadIdx.x & 31);
        if (len && start + len == nper) {
            sout[j] = x0; sout[stride + j] = x1; sout[2 * stride + j] = x2;
            sout[3 * stride + j] = y0; sout[4 * stride + j] = y1; sout[5 * stride + j] = y2;
        }
        return;
    }
    if (tid >= nstreams * nsec) return;
    uint64_t j = tid % nstreams;
    uint32_t sec = (uint32_t)(tid / nstreams);
    uint64_t start = (uint64_t)sec * seclen;
    if (start >= nper) return;
    uint64_t len = min(seclen, nper - start);
    uint32_t x0 = state[j], x1 = state[stride + j], x2 = state[2 * stride + j];
    uint32_t y0 = state[3 * stride + j], y1 = state[4 * stride + j], y2 = state[5 * stride + j];
    if (start) {
        uint32_t x[3] = { x0, x1, x2 }, y[3] = { y0, y1, y2 };
        mrg_jump_section(tab, sj, sec, start, x, y);
        x0 = x[0]; x1 = x[1]; x2 = x[2]; y0 = y[0]; y1 = y[1]; y2 = y[2];
    }
    OutT *o = out + j * nper + start;
    uint64_t i = 0;
    if (vec) {
        for (; i < len && (((j * nper + start + i) & 3u) != 0); ++i) o[i] = Cvt<OutT, true>::f(mrg_next(x0, x1, x2, y0, y1, y2));
        for (; i + 4 <= len; i += 4) {
            uint32_t a = mrg_next(x0, x1, x2, y0, y1, y2), b = mrg_next(x0, x1, x2, y0, y1, y2);
            uint32_t c = mrg_next(x0, x1, x2, y0, y1, y2), d = mrg_next(x0, x1, x2, y0, y1, y2);
            store4<OutT>(o + i, Cvt<OutT, true>::f(a), Cvt<OutT, true>::f(b), Cvt<OutT, true>::f(c), Cvt<OutT, true>::f(d));
        }
    }
    for (; i < len; ++i) o[i] = Cvt<OutT, true>::f(mrg_next(x0, x1, x2, y0, y1, y2));
    if (start + len == nper) {
        sout[j] = x0; sout[stride + j] = x1; sout[2 * stride + j] = x2;
        sout[3 * stride + j] = y0; sout[4 * stride + j] = y1; sout[5 * stride + j] = y2;
    }
}

// =========================================================== LFSR113
// tab[(c * kJumpBits + b) * 32 + i] = image of bit i under the word step of
// component c applied 2^b times.  One thread per component.
__global__ void lfsr_table_kernel(uint32_t *tab)
{
    int c = threadIdx.x;
    if (c >= 4 || blockIdx.x != 0) return;
    uint32_t col[32], sq[32];
    for (int i = 0; i < 32; ++i) col[i] = lfsr_comp_step(c, 1u << i);
    for (int b = 0; b < kJumpBits; ++b) {
        for (int i = 0; i < 32; ++i) tab[((size_t)c * kJumpBits + b) * 32 + i] = col[i];
        for (int i = 0; i < 32; ++i) sq[i] = gf2_apply(col, col[i]);
        for (int i = 0; i < 32; ++i) col[i] = sq[i];
    }
}

// Default state: 987654321 in all four words (L'Ecuyer's example seed; the paper
// prints none).  Seeded: the high 32 bits of SplitMix64 draws, redrawn while
// the top p bits of a component are all zero.
__global__ void lfsr_seed_kernel(uint32_t *base, uint64_t seed)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int P[4] = { 31, 29, 28, 25 };
    if (seed == PRAND_SEED_DEFAULT) {
        for (int c = 0; c < 4; ++c) base[c] = 987654321u;
        return;
    }
    uint64_t sm = seed;
    for (int c = 0; c < 4; ++c) {
        uint32_t w;
        do { w = (uint32_t)(splitmix64_next(sm) >> 32); } while ((w >> (32 - P[c])) == 0u);
        base[c] = w;
    }
}

// Stream j = base advanced by (first + j) * L, L of 128 bits (2^34 or 2^80);
// the exponent of up to 192 bits is exact.
__global__ void lfsr_init_kernel(const uint32_t *tab, const uint32_t *base, uint32_t *state, uint64_t first, uint64_t n,
                                 uint64_t llo, uint64_t lhi)
{
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t z[4] = { base[0], base[1], base[2], base[3] };
    uint64_t e[3];
    mul_64x128(first + j, llo, lhi, e);
    for (int w = 0; w < 3; ++w)
        for (int b = 0; e[w] && b < 64; ++b)
            if ((e[w] >> b) & 1u) lfsr_apply_bit(tab, 64 * w + b, z);
    for (int c = 0; c < 4; ++c) state[c * n + j] = z[c];
}

__global__ void lfsr_skip_kernel(const uint32_t *tab, uint32_t *state, uint64_t n, U256 off)
{
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t z[4];
    for (int c = 0; c < 4; ++c) z[c] = state[c * n + j];
    for (int b = 0; b < kJumpBits; ++b)
        if (u256_bit(off, b)) lfsr_apply_bit(tab, b, z);
    for (int c = 0; c < 4; ++c) state[c * n + j] = z[c];
}

// LFSR113 fills are bound by HBM and the store path: 256-byte row segments,
// 128-thread blocks (so the four warps' tiles stay within static shared memory).
constexpr int kLfsrRowBytes = 256;
constexpr unsigned kLfsrBlock = 128;

template <typename OutT, bool ROWS = false, typename SJ = NoSecJumps>
__global__ void __launch_bounds__(kLfsrBlock) lfsr_gen_kernel(const uint32_t *__restrict__ tab, const uint32_t *state, uint32_t *sout, uint64_t nstreams,
                                                       uint64_t stride, uint64_t nper, uint32_t nsec, uint64_t seclen,
                                                       OutT *__restrict__ out, int vec, const __grid_constant__ SJ sj)
{
    uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ROWS) {
        __shared__ __align__(16) unsigned char tiles[kLfsrBlock / 32][RowFill<OutT, kLfsrRowBytes>::TILE];
        const bool live = tid < nstreams * nsec;
        const uint64_t j = live ? tid % nstreams : 0;
        const uint64_t start = live ? (tid / nstreams) * seclen : 0;
        const uint64_t len = (live && start < nper) ? min(seclen, nper - start) : 0;
        uint32_t z0 = 0, z1 = 0, z2 = 0, z3 = 0;
        if (len) {
            z0 = state[j]; z1 = state[stride + j]; z2 = state[2 * stride + j]; z3 = state[3 * stride + j];
            if (start) {
                uint32_t z[4] = { z0, z1, z2, z3 };
                lfsr_jump_section(tab, sj, tid / nstreams, start, z);
                z0 = z[0]; z1 = z[1]; z2 = z[2]; z3 = z[3];
            }
        }
        fill_rows<OutT, kLfsrRowBytes>([&]() { return lfsr_next(z0, z1, z2, z3); }, [](uint32_t u) { return Cvt<OutT>::f(u); },
                        out + j * nper + start, len, tiles[threadIdx.x >> 5], threadIdx.x & 31);
        if (len && start + len == nper) {
            sout[j] = z0; sout[stride + j] = z1; sout[2 * stride + j] = z2; sout[3 * stride + j] = z3;
        }
        return;
    }
    if (tid >= nstreams * nsec) return;
    uint64_t j = tid % nstreams;
    uint32_t sec = (uint32_t)(tid / nstreams);
    uint64_t start = (uint64_t)sec * seclen;
    if (start >= nper) return;
    uint64_t len = min(seclen, nper - start);
    uint32_t z0 = state[j], z1 = state[stride + j], z2 = state[2 * stride + j], z3 = state[3 * stride + j];
    if (start) {
        uint32_t z[4] = { z0, z1, z2, z3 };
        lfsr_jump_section(tab, sj, sec, start, z);
        z0 = z[0]; z1 = z[1]; z2 = z[2]; z3 = z[3];
    }
    OutT *o = out + j * nper + start;
    uint64_t i = 0;
    if (vec) {
        for (; i < len && (((j * nper + start + i) & 3u) != 0); ++i) o[i] = Cvt<OutT>::f(lfsr_next(z0, z1, z2, z3));
        for (; i + 4 <= len; i += 4) {
            uint32_t a = lfsr_next(z0, z1, z2, z3), b = lfsr_next(z0, z1, z2, z3);
            uint32_t c = lfsr_next(z0, z1, z2, z3), d = lfsr_next(z0, z1, z2, z3);
            store4<OutT>(o + i, Cvt<OutT>::f(a), Cvt<OutT>::f(b), Cvt<OutT>::f(c), Cvt<OutT>::f(d));
        }
    }
    for (; i < len; ++i) o[i] = Cvt<OutT>::f(lfsr_next(z0, z1, z2, z3));
    if (start + len == nper) {
        sout[j] = z0; sout[stride + j] = z1; sout[2 * stride + j] = z2; sout[3 * stride + j] = z3;
    }
}

// =========================================================== host launchers
static unsigned grid_for(uint64_t n, unsigned block) { return (unsigned)((n + block - 1) / block); }

prand_status_t mrg_build_table(uint32_t *tab, cudaStream_t st)
{
    mrg_table_kernel<<<1, 32, 0, st>>>(tab);
    return launch_check();
}

prand_status_t lfsr_build_table(uint32_t *tab, cudaStream_t st)
{
    lfsr_table_kernel<<<1, 32, 0, st>>>(tab);
    return launch_check();
}

prand_status_t mrg_lfsr_seed(int gen, uint64_t seed, void *d_base, cudaStream_t st)
{
    if (gen == PRAND_MRG32K3A) mrg_seed_kernel<<<1, 32, 0, st>>>((uint32_t *)d_base, seed);
    else lfsr_seed_kernel<<<1, 32, 0, st>>>((uint32_t *)d_base, seed);
    return launch_check();
}

prand_status_t mrg_lfsr_init(int gen, const DevTables *T, const void *d_base, void *d_state, uint64_t first, uint64_t n,
                             const Variant &V, cudaStream_t st)
{
    const unsigned B = 128;
    if (gen == PRAND_MRG32K3A)
        mrg_init_kernel<<<grid_for(n, B), B, 0, st>>>(T->mrg, (const uint32_t *)d_base, (uint32_t *)d_state, first, n,
                                                      V.L[0], V.L[1]);
    else
        lfsr_init_kernel<<<grid_for(n, B), B, 0, st>>>(T->lfsr, (const uint32_t *)d_base, (uint32_t *)d_state, first, n,
                                                       V.L[0], V.L[1]);
    return launch_check();
}

prand_status_t mrg_lfsr_skip(int gen, const DevTables *T, void *d_state, uint64_t n, const U256 &off, cudaStream_t st)
{
    const unsigned B = 128;
    if (gen == PRAND_MRG32K3A) mrg_skip_kernel<<<grid_for(n, B), B, 0, st>>>(T->mrg, (uint32_t *)d_state, n, off);
    else lfsr_skip_kernel<<<grid_for(n, B), B, 0, st>>>(T->lfsr, (uint32_t *)d_state, n, off);
    return launch_check();
}

// Host construction of the section jumps, cached per (generator, seclen,
// nsec): M^(s seclen) for s = 1 .. nsec - 1 by square-and-multiply.
namespace {

using Gf2Mat = std::array<uint32_t, 32>;  // columns: image of bit i

Gf2Mat gf2_mul(const Gf2Mat &X, const Gf2Mat &Y)  // X Y: Y first, then X
{
    Gf2Mat R;
    for (int i = 0; i < 32; ++i) {
        uint32_t v = Y[i], r = 0;
        for (int b = 0; b < 32; ++b)
            if ((v >> b) & 1u) r ^= X[b];
        R[i] = r;
    }
    return R;
}

uint32_t lfsr_comp_step_host(int c, uint32_t z)
{
    switch (c) {
    case 0: return taus_step<31, 6, 18>(z);
    case 1: return taus_step<29, 2, 2>(z);
    case 2: return taus_step<28, 13, 7>(z);
    default: return taus_step<25, 3, 13>(z);
    }
}

using Mat3 = std::array<uint64_t, 9>;

Mat3 mat3_mul(const Mat3 &X, const Mat3 &Y, uint64_t m)
{
    Mat3 R;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            uint64_t s = 0;
            for (int k = 0; k < 3; ++k) s = (s + X[3 * i + k] * Y[3 * k + j] % m) % m;
            R[3 * i + j] = s;
        }
    return R;
}

template <typename M, typename Mul>
M mat_pow(M base, uint64_t e, M one, Mul mul)
{
    M r = one;
    while (e) {
        if (e & 1u) r = mul(r, base);
        base = mul(base, base);
        e >>= 1;
    }
    return r;
}

std::mutex g_sj_mu;
std::map<std::tuple<int, uint64_t, uint32_t>, LfsrSecJumps> g_sj_lfsr;
std::map<std::tuple<int, uint64_t, uint32_t>, MrgSecJumps> g_sj_mrg;
constexpr size_t kSecJumpCacheMax = 256;

void build_sec_jumps(uint64_t seclen, uint32_t nsec, LfsrSecJumps *out)
{
    Gf2Mat id;
    for (int i = 0; i < 32; ++i) id[i] = 1u << i;
    for (int c = 0; c < 4; ++c) {
        Gf2Mat M;
        for (int i = 0; i < 32; ++i) M[i] = lfsr_comp_step_host(c, 1u << i);
        const Gf2Mat A = mat_pow(M, seclen, id, gf2_mul);
        Gf2Mat J = A;
        for (uint32_t s = 1; s < nsec && s <= (uint32_t)kSecJumps; ++s) {
            for (int i = 0; i < 32; ++i) out->col[s - 1][c][i] = J[i];
            J = gf2_mul(J, A);
        }
    }
}

void build_sec_jumps(uint64_t seclen, uint32_t nsec, MrgSecJumps *out)
{
    const Mat3 one = { 1, 0, 0, 0, 1, 0, 0, 0, 1 };
    const Mat3 a = { 0, 1403580, kM1 - 810728, 1, 0, 0, 0, 1, 0 };
    const Mat3 b = { 527612, 0, kM2 - 1370589, 1, 0, 0, 0, 1, 0 };
    auto mul1 = [](const Mat3 &X, const Mat3 &Y) { return mat3_mul(X, Y, kM1); };
    auto mul2 = [](const Mat3 &X, const Mat3 &Y) { return mat3_mul(X, Y, kM2); };
    (void)nsec;
    Mat3 A = mat_pow(a, seclen, one, mul1), B = mat_pow(b, seclen, one, mul2);  // A^(16^j seclen)
    for (int j = 0; j < MrgSecJumps::kLevels; ++j) {
        Mat3 JA = A, JB = B;
        for (int d = 1; d < 16; ++d) {
            for (int i = 0; i < 9; ++i) {
                out->m[j][d - 1][i] = (uint32_t)JA[i];
                out->m[j][d - 1][9 + i] = (uint32_t)JB[i];
            }
            JA = mul1(JA, A);
            JB = mul2(JB, B);
        }
        A = JA;  // (A^(16^j seclen))^16
        B = JB;
    }
}

template <typename SJ>
void sec_jumps(std::map<std::tuple<int, uint64_t, uint32_t>, SJ> &cache, int gen, uint64_t seclen, uint32_t nsec,
               SJ *out)
{
    const auto key = std::make_tuple(gen, seclen, nsec);
    std::lock_guard<std::mutex> g(g_sj_mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        if (cache.size() >= kSecJumpCacheMax) cache.clear();
        SJ sj;
        std::memset(&sj, 0, sizeof sj);
        build_sec_jumps(seclen, nsec, &sj);
        it = cache.emplace(key, sj).first;
    }
    *out = it->second;
}

}  // namespace

// Sections per stream: whole waves of the kernel's resident threads (cap),
// sections no shorter than min_len outputs (256 for LFSR113, whose section
// jumps beyond the 15 tabulated ones take one table entry per set bit of the
// offset; 64 for MRG32K3A, whose take at most four products) and starting on
// multiples of 32 outputs, so the staged 128-byte row stores of every section
// fill whole cache lines.
static void pick_sections(uint64_t nstreams, uint64_t nper, uint64_t cap, uint64_t min_len, uint32_t *nsec,
                          uint64_t *seclen)
{
    const uint32_t s = pick_nsec(nstreams, cap, nper / min_len, nper);
    uint64_t len = (nper + s - 1) / s;
    len = (len + 31) & ~31ull;
    if (len == 0) len = 32;
    *seclen = len;
    *nsec = (uint32_t)((nper + len - 1) / len);
    if (*nsec == 0) *nsec = 1;
}


template <typename OutT>
static prand_status_t mrg_lfsr_gen_t(int gen, const DevTables *T, void *d_state, void *d_spare, StreamRange &R,
                                     OutT *out, uint64_t nper, cudaStream_t st)
{
    if (R.nsec == 0) {
        // size by the rows form (the other form has the same footprint or less)
        const uint64_t cap = gen == PRAND_MRG32K3A ? resident_threads<1>(mrg_gen_kernel<OutT, true>)
                                                   : resident_threads<2, kLfsrBlock>(lfsr_gen_kernel<OutT, true>);
        pick_sections(R.count, nper, cap, gen == PRAND_MRG32K3A ? 64 : 256, &R.nsec, &R.seclen);
    }
    const uint32_t nsec = R.nsec;
    const uint64_t seclen = R.seclen, nstreams = R.count;
    int vec = ((uintptr_t)out % (sizeof(OutT) == 8 ? 32 : 16)) == 0;
    const unsigned B = 256;
    uint64_t threads = nstreams * nsec;
    uint32_t *sin = (uint32_t *)d_state + R.j0, *sout = (nsec > 1 ? (uint32_t *)d_spare : (uint32_t *)d_state) + R.j0;
    // staged row stores need every row start 16-byte aligned
    constexpr uint64_t E = RowFill<OutT>::E;
    const bool rows = ((uintptr_t)out % 16) == 0 && nper % E == 0 && seclen % E == 0;
    // section jumps as one matrix per section when there are few sections
    const bool sj = nsec > 1 && (gen == PRAND_MRG32K3A ? nsec <= MrgSecJumps::kMaxSections : nsec <= (uint32_t)kSecJumps + 1);
    if (gen == PRAND_MRG32K3A) {
        const unsigned g = grid_for(threads, B);
        if (sj) {
            MrgSecJumps J;
            sec_jumps(g_sj_mrg, gen, seclen, nsec, &J);
            if (rows) mrg_gen_kernel<OutT, true, MrgSecJumps><<<g, B, 0, st>>>(T->mrg, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, J);
            else mrg_gen_kernel<OutT, false, MrgSecJumps><<<g, B, 0, st>>>(T->mrg, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, J);
        } else {
            if (rows) mrg_gen_kernel<OutT, true><<<g, B, 0, st>>>(T->mrg, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, NoSecJumps{});
            else mrg_gen_kernel<OutT><<<g, B, 0, st>>>(T->mrg, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, NoSecJumps{});
        }
    } else {
        const unsigned BL = kLfsrBlock, g = grid_for(threads, BL);
        if (sj) {
            LfsrSecJumps J;
            sec_jumps(g_sj_lfsr, gen, seclen, nsec, &J);
            if (rows) lfsr_gen_kernel<OutT, true, LfsrSecJumps><<<g, BL, 0, st>>>(T->lfsr, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, J);
            else lfsr_gen_kernel<OutT, false, LfsrSecJumps><<<g, BL, 0, st>>>(T->lfsr, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, J);
        } else {
            if (rows) lfsr_gen_kernel<OutT, true><<<g, BL, 0, st>>>(T->lfsr, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, NoSecJumps{});
            else lfsr_gen_kernel<OutT><<<g, BL, 0, st>>>(T->lfsr, sin, sout, nstreams, R.stride, nper, nsec, seclen, out, vec, NoSecJumps{});
        }
    }
    return launch_check();
}

prand_status_t mrg_lfsr_gen(int gen, const DevTables *T, void *d_state, void *d_spare, StreamRange &R, void *out,
                            int dtype, uint64_t nper, cudaStream_t st)
{
    if (dtype == PRAND_DTYPE_U32)
        return mrg_lfsr_gen_t<uint32_t>(gen, T, d_state, d_spare, R, (uint32_t *)out, nper, st);
    if (dtype == PRAND_DTYPE_F32)
        return mrg_lfsr_gen_t<float>(gen, T, d_state, d_spare, R, (float *)out, nper, st);
    return mrg_lfsr_gen_t<double>(gen, T, d_state, d_spare, R, (double *)out, nper, st);
}

}  // namespace prand

// =========================================================== no-allocation entry point
// prand_mrg32k3a_generate_u32_noalloc: the MRG32K3A u32 fill on caller-held
// states, for callers that must not allocate device memory.  Its scratch (the
// next-state buffer used when streams are split into sections, and the jump
// table the sections start from) lives in the file-scope device arrays below,
// which every GPU that loads this library keeps until the process exits.
#include <cuda.h>  // CUcontext and CUresult (the driver functions are fetched through the runtime)
#include <mutex>

namespace prand {

constexpr uint64_t kNoAllocMaxStreams = 1ull << 16;  // 65536 streams: 1.5 MB of next states
static __device__ __align__(256) uint32_t g_noalloc_next[6 * kNoAllocMaxStreams];
static __device__ __align__(256) uint32_t g_noalloc_tab[kJumpBits * 18];

__global__ void mrg_copy_words_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, uint64_t words)
{
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < words) dst[i] = src[i];
}

namespace {
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDev {
    bool ready = false;
    unsigned long long ctx = 0;  // id of the context the table was filled in (0: unknown)
    uint32_t *next = nullptr;    // device address of g_noalloc_next on this device
    uint32_t *tab = nullptr;     // device address of g_noalloc_tab on this device
};
NoAllocDev g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// The unique id of the context current on this thread, or 0 if the driver
// cannot say.  A device reset (cudaDeviceReset) replaces the primary context,
// and the arrays' contents with it, so the set-up is redone when the id
// changes.  The two driver functions are fetched through the runtime, so the
// library does not link the driver library itself.
unsigned long long current_context_id()
{
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetIdFn)f;
        cudaGetLastError();  // a missing entry point is not an error of the caller's next launch
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// With the device current: look up the device addresses of the two arrays
// (their host-side names are only stand-ins; the lookup also makes the
// device's context current on this thread) and, the first time on a device or
// after its context was replaced, fill the jump table with one launch, waited
// for so later calls on any stream see it.
prand_status_t noalloc_setup(cudaStream_t st, NoAllocDev **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return PRAND_ERR_CUDA;
    void *next = nullptr, *tab = nullptr;
    if (cudaGetSymbolAddress(&next, g_noalloc_next) != cudaSuccess || !next) return PRAND_ERR_CUDA;
    if (cudaGetSymbolAddress(&tab, g_noalloc_tab) != cudaSuccess || !tab) return PRAND_ERR_CUDA;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDev &D = g_noalloc_dev[dev];
    if (!D.ready || D.ctx != ctx || D.next != next || D.tab != tab) {
        D.ready = false;
        D.next = (uint32_t *)next;
        D.tab = (uint32_t *)tab;
        mrg_table_kernel<<<1, 32, 0, st>>>(D.tab);
        prand_status_t s = launch_check();
        if (s != PRAND_OK) return s;
        if (cudaStreamSynchronize(st) != cudaSuccess) return PRAND_ERR_CUDA;
        D.ctx = ctx;
        D.ready = true;
    }
    *out = &D;
    return PRAND_OK;
}
}  // namespace

}  // namespace prand

extern "C" prand_status_t prand_mrg32k3a_generate_u32_noalloc(uint32_t *dev_state, uint64_t n_streams, uint32_t *dev_out,
                                                               uint64_t n_per_stream, prand_stream_t stream)
{
    using namespace prand;
    if (!dev_state || !dev_out || n_streams == 0) return PRAND_ERR_ARG;
    if (n_streams > kNoAllocMaxStreams) return PRAND_ERR_ARG;  // beyond the fixed scratch
    if ((uintptr_t)dev_state % 4 || (uintptr_t)dev_out % 4) return PRAND_ERR_ALIGN;
    uint64_t total;
    if (__builtin_mul_overflow(n_streams, n_per_stream, &total) || total > (UINT64_MAX >> 2)) return PRAND_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NoAllocDev *D = nullptr;
    prand_status_t s = noalloc_setup(st, &D);
    if (s != PRAND_OK) return s;
    if (n_per_stream == 0) return PRAND_OK;
    uint32_t nsec;
    uint64_t seclen;
    // the store form of prand_generate_u32 on a handle (staged 128-byte row
    // stores whenever every row start is 16-byte aligned); sections of at least
    // 256 outputs, since this path builds no section matrices (that would
    // allocate host memory) and jumps by one table entry per set bit
    pick_sections(n_streams, n_per_stream, resident_threads<1>(mrg_gen_kernel<uint32_t, true>), 256, &nsec, &seclen);
    int vec = ((uintptr_t)dev_out % 16) == 0;
    constexpr uint64_t E = RowFill<uint32_t>::E;
    const bool rows = vec && n_per_stream % E == 0 && seclen % E == 0;
    const unsigned B = 256;
    const unsigned grid = grid_for(n_streams * nsec, B);
    uint32_t *sout = nsec > 1 ? D->next : dev_state;
    if (rows)
        mrg_gen_kernel<uint32_t, true><<<grid, B, 0, st>>>(D->tab, dev_state, sout, n_streams, n_streams, n_per_stream,
                                                           nsec, seclen, dev_out, vec, NoSecJumps{});
    else
        mrg_gen_kernel<uint32_t><<<grid, B, 0, st>>>(D->tab, dev_state, sout, n_streams, n_streams, n_per_stream, nsec,
                                                     seclen, dev_out, vec, NoSecJumps{});
    if ((s = launch_check()) != PRAND_OK) return s;
    if (nsec > 1) {
        mrg_copy_words_kernel<<<grid_for(6 * n_streams, B), B, 0, st>>>(D->next, dev_state, 6 * n_streams);
        if ((s = launch_check()) != PRAND_OK) return s;
    }
    return PRAND_OK;
}
