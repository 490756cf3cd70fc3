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

struct Reducer {
    // phi shifted left by 0..63 bits
    std::vector<Poly> sh;
    explicit Reducer(const Poly &phi)
    {
        sh.assign(64, Poly((size_t)kW, 0));
        for (int s = 0; s < 64; ++s)
            for (int j = 0; j <= kDeg; ++j)
                if (getb(phi, j)) flipb(sh[(size_t)s], j + s);
    }
    // r (degree < 2*kDeg) mod phi, in place
    void reduce(Poly &r) const
    {
        for (int i = 2 * kDeg; i >= kDeg; --i) {
            if (!getb(r, i)) continue;
            int s = i - kDeg, w = s >> 6;
            const Poly &P = sh[(size_t)(s & 63)];
            const int nw = (kDeg + 64) / 64 + 1;
            for (int k = 0; k < nw && w + k < kW; ++k) r[(size_t)(w + k)] ^= P[(size_t)k];
        }
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

// a * b (degrees < kDeg, carry-less) into out, reduced mod phi.  For every set
// bit of b, a copy of a shifted by that bit is added: the 64 shifts of a within
// a word are made once, so each set bit costs one pass over a's words.
void mul_into(const Poly &a, const Poly &b, Poly &out, const Reducer &red)
{
    const int nw = (kDeg + 63) / 64;  // words of a reduced polynomial
    std::vector<Poly> sh(64, Poly((size_t)nw + 1, 0));
    for (int s = 0; s < 64; ++s)
        for (int w = 0; w <= nw; ++w) {
            const uint64_t lo = w < nw ? a[(size_t)w] : 0, prev = w > 0 ? a[(size_t)(w - 1)] : 0;
            sh[(size_t)s][(size_t)w] = s ? (lo << s) | (prev >> (64 - s)) : lo;
        }
    std::fill(out.begin(), out.end(), 0ull);
    for (int w = 0; w < nw; ++w) {
        uint64_t v = b[(size_t)w];
        while (v) {
            const int s = __builtin_ctzll(v);
            v &= v - 1;
            const Poly &A = sh[(size_t)s];
            for (int k = 0; k <= nw; ++k) out[(size_t)(w + k)] ^= A[(size_t)k];
        }
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
    g_win.assign((size_t)kMtWinPositions * 16 * kMtPolyWords, 0u);
    const Reducer red(g_phi);
    // position i: x^(d 2^(kMtStreamShift + 4 i)) mod phi for digits d = 1..15;
    // the powers of two are stored already, the other digits are one product each
    auto position = [&](int i) {
        std::vector<Poly> P(16);
        for (int t = 0; t < 4; ++t) P[(size_t)(1 << t)] = from_words(pw + (size_t)(kMtStreamShift + 4 * i + t) * kMtPolyWords);
        for (int d = 3; d < 16; ++d) {
            if ((d & (d - 1)) == 0) continue;
            const int hi = 1 << (31 - __builtin_clz((unsigned)d));
            P[(size_t)d].assign((size_t)kW, 0);
            mul_into(P[(size_t)hi], P[(size_t)(d - hi)], P[(size_t)d], red);
        }
        for (int d = 1; d < 16; ++d) {
            uint32_t *dst = g_win.data() + ((size_t)i * 16 + d) * kMtPolyWords;
            for (int k = 0; k < kMtPolyWords / 2; ++k) {
                dst[2 * k] = (uint32_t)P[(size_t)d][(size_t)k];
                dst[2 * k + 1] = (uint32_t)(P[(size_t)d][(size_t)k] >> 32);
            }
        }
    };
    std::vector<std::thread> th;
    for (int i = 0; i < kMtWinPositions; ++i) th.emplace_back(position, i);
    for (std::thread &t : th) t.join();
    g_win_ok = true;
}
}  // namespace

const uint32_t *mt_host_window_polys()
{
    std::call_once(g_win_once, compute_window);
    return g_win_ok ? g_win.data() : nullptr;
}

}  // namespace prand
