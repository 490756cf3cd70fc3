// Host precomputation for the MT19937 jump (Sec. 5.4): the characteristic
// polynomial phi of the state transition and the polynomials x^(2^b) mod phi,
// b = 0..511 (the paper stores the same family "v = 2^n, n = 0..511").
//
// phi is the minimal polynomial of one output bit sequence, found by the
// Berlekamp-Massey algorithm over GF(2) on 2 * 19937 + 64 bits (degree 19937,
// because phi is primitive).  The squaring chain then costs 511 squarings
// modulo phi.  Like the paper's stored coefficients, this is computed once (per
// process) and uploaded to the device, where the per-stream jumps run.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "prand_internal.h"

namespace prand {
namespace {

constexpr int kDeg = kMtDeg;
constexpr int kW = (2 * kDeg + 64 + 63) / 64 + 2;  // words of a working polynomial

using Poly = std::vector<uint64_t>;

inline int getb(const Poly &p, int i) { return (int)((p[(size_t)i >> 6] >> (i & 63)) & 1u); }
inline void flipb(Poly &p, int i) { p[(size_t)i >> 6] ^= 1ull << (i & 63); }

// Bit 31 of the untempered recurrence words x_624, x_625, ... from init_genrand(1).
std::vector<uint8_t> mt_bit_sequence(int nbits)
{
    uint32_t mt[kMtN];
    mt[0] = 1u;
    for (uint32_t i = 1; i < (uint32_t)kMtN; ++i) mt[i] = 1812433253u * (mt[i - 1] ^ (mt[i - 1] >> 30)) + i;
    std::vector<uint8_t> s((size_t)nbits);
    int h = 0;
    for (int n = 0; n < nbits; ++n) {
        uint32_t y = (mt[h] & 0x80000000u) | (mt[(h + 1) % kMtN] & 0x7FFFFFFFu);
        uint32_t x = mt[(h + kMtM) % kMtN] ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
        mt[h] = x;
        h = (h + 1) % kMtN;
        s[(size_t)n] = (uint8_t)(x >> 31);
    }
    return s;
}

// Word-packed Berlekamp-Massey.  The sequence is stored reversed so that the
// discrepancy sum over s_{n-i} is an AND-parity against a shifted bit window.
int berlekamp_massey(const std::vector<uint8_t> &s, Poly &C)
{
    const int N = (int)s.size();
    const int W = N / 64 + 3;
    Poly R((size_t)W + 2, 0);  // R bit k = s[N-1-k]
    for (int k = 0; k < N; ++k)
        if (s[(size_t)(N - 1 - k)]) R[(size_t)k >> 6] |= 1ull << (k & 63);
    C.assign((size_t)W, 0);
    Poly B((size_t)W, 0), T;
    C[0] = 1; B[0] = 1;
    int L = 0, m = 1;
    for (int n = 0; n < N; ++n) {
        // d = sum_{i=0..L} c_i s_{n-i} = parity(C & (R >> (N-1-n))) over bits 0..L
        int off = N - 1 - n, q = off >> 6, r = off & 63;
        int words = (L >> 6) + 1;
        uint64_t acc = 0;
        for (int w = 0; w < words; ++w) {
            uint64_t lo = R[(size_t)(w + q)], hi = R[(size_t)(w + q + 1)];
            uint64_t win = r ? ((lo >> r) | (hi << (64 - r))) : lo;
            acc ^= C[(size_t)w] & win;
        }
        // bits of C above L are zero, so no masking is needed
        int d = __builtin_parityll(acc);
        if (!d) { ++m; continue; }
        auto xor_shifted = [&](Poly &dst, const Poly &src, int sh) {
            int qs = sh >> 6, rs = sh & 63;
            for (int w = W - 1; w >= qs; --w) {
                uint64_t v = src[(size_t)(w - qs)] << rs;
                if (rs && w - qs - 1 >= 0) v |= src[(size_t)(w - qs - 1)] >> (64 - rs);
                dst[(size_t)w] ^= v;
            }
        };
        if (2 * L <= n) {
            T = C;
            xor_shifted(C, B, m);
            L = n + 1 - L;
            B = T;
            m = 1;
        } else {
            xor_shifted(C, B, m);
            ++m;
        }
    }
    return L;
}

// Reduction modulo phi eight coefficients at a time.  For every byte t, P_t is
// the multiple of phi whose coefficients kDeg .. kDeg + 7 are the bits of t and
// whose higher ones vanish (t x^kDeg minus the multiple is the remainder of t
// x^kDeg).  XORing P_t x^(8 c) into r, with t the byte of r at kDeg + 8 c,
// clears that byte; bytes are cleared from the top down.  Eight bytes are
// cleared per pass over r: their t are found one after another from r and
// the bytes that the P_t above them leave just below their own top (tables
// below[1..7]), and the eight shifted P_t are then added in one pass.  Shifts
// by whole bytes are byte offsets (bit i of a polynomial is bit i % 8 of byte
// i / 8 in the little-endian word arrays on both host architectures).
static_assert(__BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__, "byte offsets assume little-endian words");

inline uint64_t ld64(const unsigned char *p) { uint64_t v; memcpy(&v, p, 8); return v; }
inline void st64(unsigned char *p, uint64_t v) { memcpy(p, &v, 8); }

struct Reducer {
    static constexpr int kPB = ((kDeg + 8 + 7) / 8 + 7) / 8 * 8;  // bytes of P_t, rounded to words
    static constexpr int kRow = 8 + kPB + 16;                      // zero bytes before and after
    std::vector<unsigned char> tab;                                 // [256][kRow]
    uint8_t below[8][256];                                          // below[k][t]: P_t bits kDeg-8k .. kDeg-8k+7
    explicit Reducer(const Poly &phi)
    {
        const int nw = kPB / 8 + 1;
        std::vector<Poly> phs(8, Poly((size_t)nw, 0));  // phi x^k, k = 0..7
        for (int k = 0; k < 8; ++k)
            for (int j = 0; j <= kDeg; ++j)
                if (getb(phi, j)) flipb(phs[(size_t)k], j + k);
        tab.assign((size_t)256 * kRow, 0);
        Poly T((size_t)nw, 0);
        for (int t = 0; t < 256; ++t) {
            std::fill(T.begin(), T.end(), 0ull);
            for (int k = 0; k < 8; ++k)
                if ((t >> k) & 1) flipb(T, kDeg + k);
            for (int k = 7; k >= 0; --k)
                if (getb(T, kDeg + k))
                    for (int w = 0; w < nw; ++w) T[(size_t)w] ^= phs[(size_t)k][(size_t)w];
            // T is now the remainder; P_t = T + t x^kDeg
            for (int k = 0; k < 8; ++k)
                if ((t >> k) & 1) flipb(T, kDeg + k);
            memcpy(tab.data() + (size_t)t * kRow + 8, T.data(), (size_t)kPB);
            for (int k = 0; k < 8; ++k) {
                uint8_t b = 0;
                for (int i = 0; i < 8; ++i) b |= (uint8_t)(getb(T, kDeg - 8 * k + i) << i);
                below[k][t] = b;
            }
        }
    }
    static uint8_t byte_at(const unsigned char *r, int pos)  // bits pos .. pos + 7
    {
        return (uint8_t)(((unsigned)r[pos >> 3] | ((unsigned)r[(pos >> 3) + 1] << 8)) >> (pos & 7));
    }
    // clears bytes c0 .. c0 + n - 1 (n <= 8) of the part above kDeg
    void group(unsigned char *r, int c0, int n) const
    {
        uint8_t t[8] = { 0, 0, 0, 0, 0, 0, 0, 0 };
        for (int j = n - 1; j >= 0; --j) {
            uint8_t b = byte_at(r, kDeg + 8 * (c0 + j));
            for (int k = j + 1; k < n; ++k) b ^= below[k - j][t[k]];
            t[j] = b;
        }
        const unsigned char *P[8];
        for (int j = 0; j < 8; ++j) P[j] = tab.data() + (size_t)t[j] * kRow + 8 - j;
        unsigned char *R = r + c0;
        for (int i = 0; i < kPB + 8; i += 8)
            st64(R + i, ld64(R + i) ^ ld64(P[0] + i) ^ ld64(P[1] + i) ^ ld64(P[2] + i) ^ ld64(P[3] + i) ^ ld64(P[4] + i) ^
                            ld64(P[5] + i) ^ ld64(P[6] + i) ^ ld64(P[7] + i));
    }
    // r (degree <= 2 kDeg, kW words) mod phi, in place
    void reduce(Poly &r) const
    {
        unsigned char *rb = reinterpret_cast<unsigned char *>(r.data());
        int c = kDeg / 8;  // top byte
        for (; c >= 7; c -= 8) group(rb, c - 7, 8);
        if (c >= 0) group(rb, 0, c + 1);
    }
};

// square of a polynomial of degree < kDeg: bit i -> bit 2i (spread each 32-bit half)
void square_into(const Poly &a, Poly &out)
{
    std::fill(out.begin(), out.end(), 0ull);
    const int nw = (kDeg + 63) / 64;
    for (int w = 0; w < nw; ++w) {
        uint64_t v = a[(size_t)w];
        for (int half = 0; half < 2; ++half) {
            uint64_t x = (v >> (32 * half)) & 0xFFFFFFFFull;
            x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
            x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
            x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
            x = (x | (x << 2)) & 0x3333333333333333ull;
            x = (x | (x << 1)) & 0x5555555555555555ull;
            out[(size_t)(2 * w + half)] = x;
        }
    }
}

// a * b (degrees < kDeg, carry-less) into out, reduced mod phi.  The products
// of a with every byte t are tabulated (each is the previous one with the
// lowest set bit of t removed, plus a x^k for that bit); eight bytes of b are
// then added per pass, each as its row at the byte's offset.
void mul_into(const Poly &a, const Poly &b, Poly &out, const Reducer &red)
{
    constexpr int kPB = Reducer::kPB, kRow = Reducer::kRow, nw = kPB / 8;
    std::vector<Poly> ash(8, Poly((size_t)nw, 0));  // a x^k, k = 0..7 (degree < kDeg + 7)
    for (int k = 0; k < 8; ++k)
        for (int w = 0; w < nw; ++w) {
            const uint64_t lo = a[(size_t)w], prev = w > 0 ? a[(size_t)(w - 1)] : 0;
            ash[(size_t)k][(size_t)w] = k ? (lo << k) | (prev >> (64 - k)) : lo;
        }
    std::vector<unsigned char> rows((size_t)256 * kRow, 0);
    for (int t = 1; t < 256; ++t) {
        const unsigned char *src = rows.data() + (size_t)(t & (t - 1)) * kRow + 8;
        unsigned char *dst = rows.data() + (size_t)t * kRow + 8;
        const uint64_t *A = ash[(size_t)__builtin_ctz((unsigned)t)].data();
        for (int w = 0; w < nw; ++w) st64(dst + 8 * w, ld64(src + 8 * w) ^ A[w]);
    }
    std::fill(out.begin(), out.end(), 0ull);
    const unsigned char *bb = reinterpret_cast<const unsigned char *>(b.data());
    unsigned char *ob = reinterpret_cast<unsigned char *>(out.data());
    for (int g = 0; g < (kDeg + 7) / 8; g += 8) {
        const unsigned char *P[8];
        for (int j = 0; j < 8; ++j) P[j] = rows.data() + (size_t)bb[g + j] * kRow + 8 - j;
        unsigned char *R = ob + g;
        for (int i = 0; i < kPB + 8; i += 8)
            st64(R + i, ld64(R + i) ^ ld64(P[0] + i) ^ ld64(P[1] + i) ^ ld64(P[2] + i) ^ ld64(P[3] + i) ^ ld64(P[4] + i) ^
                            ld64(P[5] + i) ^ ld64(P[6] + i) ^ ld64(P[7] + i));
    }
    red.reduce(out);
}

std::vector<uint32_t> g_polys;
std::once_flag g_once;
bool g_ok = false;
Poly g_phi;  // kept for the window table

void compute()
{
    std::vector<uint8_t> s = mt_bit_sequence(2 * kDeg + 64);
    Poly C;
    int L = berlekamp_massey(s, C);
    if (L != kDeg) return;
    Poly phi((size_t)kW, 0);
    for (int j = 0; j <= L; ++j)
        if (getb(C, L - j)) flipb(phi, j);
    g_phi = phi;
    Reducer red(phi);
    g_polys.assign((size_t)kMtPolyCount * kMtPolyWords, 0u);
    Poly cur((size_t)kW, 0), sq((size_t)kW, 0);
    cur[0] = 2;  // x
    for (int b = 0; b < kMtPolyCount; ++b) {
        uint32_t *dst = g_polys.data() + (size_t)b * kMtPolyWords;
        for (int k = 0; k < kMtPolyWords / 2; ++k) {
            dst[2 * k] = (uint32_t)cur[(size_t)k];
            dst[2 * k + 1] = (uint32_t)(cur[(size_t)k] >> 32);
        }
        if (b + 1 < kMtPolyCount) {
            square_into(cur, sq);
            red.reduce(sq);
            std::fill(cur.begin(), cur.end(), 0ull);
            for (int k = 0; k < (kDeg + 63) / 64; ++k) cur[(size_t)k] = sq[(size_t)k];
        }
    }
    g_ok = true;
}

}  // namespace

const uint32_t *mt_host_pow2_polys()
{
    std::call_once(g_once, compute);
    return g_ok ? g_polys.data() : nullptr;
}

namespace {
std::vector<uint32_t> g_win;
std::once_flag g_win_once;
bool g_win_ok = false;

Poly from_words(const uint32_t *w)
{
    Poly p((size_t)kW, 0);
    for (int k = 0; k < kMtPolyWords / 2; ++k) p[(size_t)k] = (uint64_t)w[2 * k] | ((uint64_t)w[2 * k + 1] << 32);
    return p;
}

void compute_window()
{
    const uint32_t *pw = mt_host_pow2_polys();
    if (!pw) return;
    constexpr int D = kMtWinDigits;
    g_win.assign((size_t)kMtWinPositions * D * kMtPolyWords, 0u);
    const Reducer red(g_phi);
    // P[i][d] = x^(d 2^(kMtStreamShift + 8 i)) mod phi.  The powers of two are
    // stored already; every other digit d is one product, of its highest bit
    // 2^b and of d - 2^b < 2^b, so the digits with the same highest bit form a
    // wave whose products are independent and run on all host threads.
    std::vector<std::vector<Poly>> P((size_t)kMtWinPositions, std::vector<Poly>((size_t)D));
    for (int i = 0; i < kMtWinPositions; ++i)
        for (int t = 0; t < kMtWinBits; ++t)
            P[(size_t)i][(size_t)(1 << t)] = from_words(pw + (size_t)(kMtStreamShift + kMtWinBits * i + t) * kMtPolyWords);
    const unsigned hw = std::thread::hardware_concurrency();
    const int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 64u));
    for (int b = 1; b < kMtWinBits; ++b) {
        std::vector<std::pair<int, int>> items;  // (position, digit) of this wave
        for (int i = 0; i < kMtWinPositions; ++i)
            for (int d = (1 << b) + 1; d < (2 << b); ++d) items.emplace_back(i, d);
        std::atomic<size_t> next(0);
        auto work = [&]() {
            for (size_t k; (k = next.fetch_add(1)) < items.size();) {
                const int i = items[k].first, d = items[k].second;
                Poly &out = P[(size_t)i][(size_t)d];
                out.assign((size_t)kW, 0);
                mul_into(P[(size_t)i][(size_t)(1 << b)], P[(size_t)i][(size_t)(d - (1 << b))], out, red);
            }
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nth && (size_t)t < items.size(); ++t) th.emplace_back(work);
        work();
        for (std::thread &t : th) t.join();
    }
    for (int i = 0; i < kMtWinPositions; ++i)
        for (int d = 1; d < D; ++d) {
            uint32_t *dst = g_win.data() + ((size_t)i * D + d) * kMtPolyWords;
            const Poly &src = P[(size_t)i][(size_t)d];
            for (int k = 0; k < kMtPolyWords / 2; ++k) {
                dst[2 * k] = (uint32_t)src[(size_t)k];
                dst[2 * k + 1] = (uint32_t)(src[(size_t)k] >> 32);
            }
        }
    g_win_ok = true;
}
}  // namespace

const uint32_t *mt_host_window_polys()
{
    std::call_once(g_win_once, compute_window);
    return g_win_ok ? g_win.data() : nullptr;
}

}  // namespace prand
