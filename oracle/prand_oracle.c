/*
 * prand_oracle.c -- plain, slow, single-threaded CPU oracle for the eleven
 * PRAND generators (Barash & Shchur, "PRAND: GPU accelerated parallel random
 * number generation library", CPC 185 (2014) 1343).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, imports or calls
 * this file.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant generator
 * with the CUDA path; it is written straight from the definitions below.
 *
 * Every output is an exact integer sequence, so the oracle computes it the
 * plain way: one recurrence step at a time, exact big-integer jump offsets,
 * and matrix / polynomial powers by square-and-multiply.
 *
 * What each part follows:
 *   MT19937   Matsumoto & Nishimura 1998 (the paper's [MT19937], Sec. 4, 5.4).
 *             Seeding: init_genrand for 32-bit seeds, init_by_array {lo,hi}
 *             for wider seeds (reading; Sec. 7.1 does not print seeds).
 *             Jump: Sec. 5.4, eq. (g_v): A^v Y = sum_i a_i A^(i-1) Y with
 *             g_v = x^v mod phi, phi from Berlekamp-Massey.
 *   MRG32K3A  Sec. 5.2 (matrices A, B, a, b, c, d, m1, m2); jump by A^n, B^n.
 *             Output: the printed "(x_n + y_n) mod g" is garbled (g is not
 *             defined for MRG32K3A); reading: z = (x_n - y_n) mod m1 with 0
 *             replaced by m1, as in the cited original.
 *   LFSR113   Sec. 5.3, eqs. (lfsrRel1), (lfsrOutput), four components with
 *             (p,q,s) = (31,6,18), (29,2,2), (28,13,7), (25,3,13); combined
 *             by XOR of the component words (reading of "combination").
 *   GM/GQ     Sec. 5.1, eq. (rec1) with (k,q,g,v) of Table 2; jump by the
 *             2x2 matrix power (equivalent to eqs. (rec2), (rec3)).
 *             Ensemble size s, output map, seeding and block lengths are
 *             readings (the paper gives only k, q, g, v): see gm_params().
 *   Floats    Sec. 7.3 says only "uniform in [0,1)"; reading:
 *             f32 = (u >> 8) * 2^-24, f64 = u * 2^-32, MRG f64 = z * RN(1/(m1+1)).
 *
 *   Variants  Table 4 lists up to three stream-initialisation variants per
 *             generator (short / medium / long sequences); each is the pair
 *             (number of sequences, block length L) of orc_variant(); the
 *             GM/GQ ensemble of a variant spaces its points by that variant's
 *             N_max L (reading); LFSR113 long: L = 2^80 (reading: >= 1e24).
 *
 *   Spaced    Table 3 tests the generators on the subsequence that skips
 *             2^n values at each step; orc_stream_spaced() gives stream k of
 *             the layout whose streams start k * 2^n outputs after the base,
 *             so output 0 of streams 0, 1, 2, ... is that subsequence.
 *   Tests     The statistical tests applied to such subsequences (the
 *             paper runs TestU01; this build carries three classical tests
 *             from Knuth, TAOCP vol. 2, Sec. 3.3.2): frequency (cells of the
 *             top b bits), serial (non-overlapping pairs, cells of the top b
 *             bits of each word), gap (Algorithm G's gap lengths for a word
 *             range [lo, hi)).  The oracle computes the cell counts.
 *
 * Parity unpinned (readings of gaps in the paper, pinned only by invariants):
 *   the GM/GQ output map, ensemble size, seeding and block lengths; the MRG32K3A
 *   output map and default state; the LFSR113 default state and combination;
 *   the float conversions' exact form; the variants' block lengths.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Generator ids (same order as the library's public enum). */
enum {
    O_MT19937 = 0, O_MRG32K3A = 1, O_LFSR113 = 2, O_GM19 = 3, O_GM29 = 4,
    O_GM31 = 5, O_GM55 = 6, O_GM61 = 7, O_GQ58_1 = 8, O_GQ58_3 = 9, O_GQ58_4 = 10
};

#define SEED_DEFAULT UINT64_MAX
#define NBIG 8 /* 512-bit little-endian jump offsets */

/* ------------------------------------------------------------------ */
/* Small helpers: SplitMix64 (Steele, Lea & Flood 2014), big offsets.  */
/* ------------------------------------------------------------------ */

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One SplitMix64 output from the caller's 64-bit state (exported for its pin). */
uint64_t orc_splitmix64(uint64_t *s) { return splitmix64(s); }

static int big_bit(const uint64_t *e, int i) { return (int)((e[i >> 6] >> (i & 63)) & 1u); }

static int big_nbits(const uint64_t *e)
{
    for (int w = NBIG - 1; w >= 0; --w)
        if (e[w]) return 64 * w + 64 - __builtin_clzll(e[w]);
    return 0;
}

/* r = a * m  (a: NBIG words, m: 64-bit). */
static void big_mul_u64(uint64_t *r, const uint64_t *a, uint64_t m)
{
    u128 carry = 0;
    for (int i = 0; i < NBIG; ++i) {
        u128 t = (u128)a[i] * m + carry;
        r[i] = (uint64_t)t;
        carry = t >> 64;
    }
}

/* ------------------------------------------------------------------ */
/* Float conversions (reading of Sec. 7.3, "uniform in [0,1)").        */
/* ------------------------------------------------------------------ */

float orc_u32_to_f32(uint32_t u) { return (float)(u >> 8) * 0x1p-24f; }
double orc_u32_to_f64(uint32_t u) { return (double)u * 0x1p-32; }
/* MRG32K3A: z in [1, m1] times the correctly rounded 1/(m1+1), one RN multiply. */
static const double MRG_NORM = 1.0 / 4294967088.0;
double orc_mrg_to_f64(uint32_t z) { return (double)z * MRG_NORM; }

/* The three float maps over an array (kind 0: f32, 1: f64, 2: MRG32K3A f64),
 * one value at a time with the functions above. */
void orc_convert(const uint32_t *in, uint64_t n, int kind, void *out)
{
    for (uint64_t i = 0; i < n; ++i) {
        if (kind == 0) ((float *)out)[i] = orc_u32_to_f32(in[i]);
        else if (kind == 1) ((double *)out)[i] = orc_u32_to_f64(in[i]);
        else ((double *)out)[i] = orc_mrg_to_f64(in[i]);
    }
}

/* ================================================================== */
/* MT19937 (Matsumoto & Nishimura 1998; Sec. 5.4)                      */
/* ================================================================== */

#define MT_N 624
#define MT_M 397
#define MT_A 0x9908B0DFu
#define MT_UPPER 0x80000000u
#define MT_LOWER 0x7FFFFFFFu
#define MT_DEG 19937
#define MT_PW 312 /* 64-bit words for a polynomial of degree < 19937 (19968 bits) */

typedef struct { uint32_t mt[MT_N]; uint32_t idx; } mt_state;

static void mt_init_genrand(mt_state *s, uint32_t seed)
{
    s->mt[0] = seed;
    for (uint32_t i = 1; i < MT_N; ++i)
        s->mt[i] = 1812433253u * (s->mt[i - 1] ^ (s->mt[i - 1] >> 30)) + i;
    s->idx = MT_N;
}

static void mt_init_by_array(mt_state *s, const uint32_t *key, int len)
{
    mt_init_genrand(s, 19650218u);
    int i = 1, j = 0;
    for (int k = (MT_N > len ? MT_N : len); k; --k) {
        s->mt[i] = (s->mt[i] ^ ((s->mt[i - 1] ^ (s->mt[i - 1] >> 30)) * 1664525u)) + key[j] + (uint32_t)j;
        ++i; ++j;
        if (i >= MT_N) { s->mt[0] = s->mt[MT_N - 1]; i = 1; }
        if (j >= len) j = 0;
    }
    for (int k = MT_N - 1; k; --k) {
        s->mt[i] = (s->mt[i] ^ ((s->mt[i - 1] ^ (s->mt[i - 1] >> 30)) * 1566083941u)) - (uint32_t)i;
        ++i;
        if (i >= MT_N) { s->mt[0] = s->mt[MT_N - 1]; i = 1; }
    }
    s->mt[0] = 0x80000000u;
    s->idx = MT_N;
}

static void mt_seed(mt_state *s, uint64_t seed)
{
    if (seed == SEED_DEFAULT) { mt_init_genrand(s, 5489u); return; }
    if (seed <= 0xFFFFFFFFull) { mt_init_genrand(s, (uint32_t)seed); return; }
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    mt_init_by_array(s, key, 2);
}

/* One word of the linear recurrence: x_{t+624} = x_{t+397} ^ twist(x_t^u | x_{t+1}^l). */
static uint32_t mt_recur(uint32_t xt, uint32_t xt1, uint32_t xt397)
{
    uint32_t y = (xt & MT_UPPER) | (xt1 & MT_LOWER);
    return xt397 ^ (y >> 1) ^ ((y & 1u) ? MT_A : 0u);
}

static uint32_t mt_temper(uint32_t y)
{
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

static uint32_t mt_next(mt_state *s)
{
    if (s->idx >= MT_N) {
        for (int k = 0; k < MT_N; ++k)
            s->mt[k] = mt_recur(s->mt[k], s->mt[(k + 1) % MT_N], s->mt[(k + MT_M) % MT_N]);
        s->idx = 0;
    }
    return mt_temper(s->mt[s->idx++]);
}

/* --- GF(2)[x] polynomials, bit i = coefficient of x^i. --- */

static uint64_t mt_phi[MT_PW + 2];   /* characteristic polynomial, degree 19937 */
static int mt_phi_ready = 0;

/* Berlekamp-Massey over GF(2) on n bits s[0..n-1] (one byte per bit).
 * Returns the linear complexity L and the connection polynomial c[0..L]
 * (c[0] = 1) with s_t + sum_{i=1..L} c_i s_{t-i} = 0. */
static int bm_gf2(const uint8_t *s, int n, uint8_t *c)
{
    uint8_t *b = calloc((size_t)n + 1, 1), *t = calloc((size_t)n + 1, 1);
    memset(c, 0, (size_t)n + 1);
    c[0] = 1; b[0] = 1;
    int L = 0, m = -1;
    for (int i = 0; i < n; ++i) {
        uint8_t d = s[i];
        for (int j = 1; j <= L; ++j) d ^= (uint8_t)(c[j] & s[i - j]);
        if (!d) continue;
        memcpy(t, c, (size_t)n + 1);
        int shift = i - m;
        for (int j = 0; j + shift <= n; ++j) c[j + shift] ^= b[j];
        if (2 * L <= i) { L = i + 1 - L; m = i; memcpy(b, t, (size_t)n + 1); }
    }
    free(b); free(t);
    return L;
}

/* phi(x) = x^L c(1/x): the characteristic polynomial of the state transition
 * (its degree must be 19937; the linear complexity of one output bit). */
static void mt_compute_phi(void)
{
    if (mt_phi_ready) return;
    const int n = 2 * MT_DEG + 64;
    uint8_t *bits = malloc((size_t)n), *c = malloc((size_t)n + 1);
    mt_state s; mt_init_genrand(&s, 5489u);
    for (int i = 0; i < n; ++i) bits[i] = (uint8_t)(mt_next(&s) & 1u);
    int L = bm_gf2(bits, n, c);
    memset(mt_phi, 0, sizeof mt_phi);
    if (L == MT_DEG)
        for (int j = 0; j <= L; ++j)
            if (c[L - j]) mt_phi[j >> 6] |= 1ull << (j & 63);
    free(bits); free(c);
    mt_phi_ready = (L == MT_DEG);
}

int orc_mt_charpoly(uint64_t *out /* MT_PW+1 words */)
{
    mt_compute_phi();
    memcpy(out, mt_phi, (MT_PW + 1) * sizeof(uint64_t));
    return mt_phi_ready ? MT_DEG : -1;
}

/* phi shifted left by 0..63 bits, so reducing one bit is an aligned XOR. */
static uint64_t mt_phi_sh[64][MT_PW + 2];
static int mt_phi_sh_ready = 0;

static void mt_prepare_shifts(void)
{
    if (mt_phi_sh_ready) return;
    mt_compute_phi();
    for (int sh = 0; sh < 64; ++sh) {
        memset(mt_phi_sh[sh], 0, sizeof mt_phi_sh[sh]);
        for (int j = 0; j <= MT_DEG; ++j)
            if ((mt_phi[j >> 6] >> (j & 63)) & 1u) {
                int k = j + sh;
                mt_phi_sh[sh][k >> 6] |= 1ull << (k & 63);
            }
    }
    mt_phi_sh_ready = 1;
}

/* r (2*MT_PW+2 words, degree < 2*19937) reduced mod phi in place. */
static void poly_reduce(uint64_t *r)
{
    for (int i = 2 * MT_DEG; i >= MT_DEG; --i) {
        if (!((r[i >> 6] >> (i & 63)) & 1u)) continue;
        int s = i - MT_DEG, w = s >> 6, sh = s & 63;
        for (int k = 0; k < MT_PW + 2 && w + k < 2 * MT_PW + 2; ++k) r[w + k] ^= mt_phi_sh[sh][k];
    }
}

/* a <- a^2 mod phi (a has MT_PW+1 words on entry and exit). */
static void poly_sqr_mod(uint64_t *a)
{
    uint64_t r[2 * MT_PW + 2];
    memset(r, 0, sizeof r);
    for (int i = 0; i < MT_DEG; ++i)
        if ((a[i >> 6] >> (i & 63)) & 1u) r[(2 * i) >> 6] |= 1ull << ((2 * i) & 63);
    poly_reduce(r);
    memcpy(a, r, (MT_PW + 1) * sizeof(uint64_t));
}

/* a <- a * x mod phi. */
static void poly_mulx_mod(uint64_t *a)
{
    uint64_t r[2 * MT_PW + 2];
    memset(r, 0, sizeof r);
    for (int i = 0; i < MT_DEG; ++i)
        if ((a[i >> 6] >> (i & 63)) & 1u) r[(i + 1) >> 6] |= 1ull << ((i + 1) & 63);
    poly_reduce(r);
    memcpy(a, r, (MT_PW + 1) * sizeof(uint64_t));
}

/* g = x^e mod phi, left-to-right square-and-multiply (Sec. 5.4). */
void orc_mt_jump_poly(const uint64_t *e, uint64_t *g /* MT_PW+1 words */)
{
    mt_prepare_shifts();
    memset(g, 0, (MT_PW + 1) * sizeof(uint64_t));
    g[0] = 1;
    for (int b = big_nbits(e) - 1; b >= 0; --b) {
        poly_sqr_mod(g);
        if (big_bit(e, b)) poly_mulx_mod(g);
    }
}

/* g = x^(2^k) mod phi by k squarings of x (period checks reach k = 19937). */
void orc_mt_x_pow2k(int k, uint64_t *g /* MT_PW+1 words */)
{
    mt_prepare_shifts();
    memset(g, 0, (MT_PW + 1) * sizeof(uint64_t));
    g[0] = 2;
    for (int i = 0; i < k; ++i) poly_sqr_mod(g);
}

/* Cache of x^(2^b) mod phi, b = 0..511 (the paper's stored v = 2^n family). */
static uint64_t *mt_pow2_polys[512];

static const uint64_t *mt_pow2_poly(int b)
{
    mt_prepare_shifts();
    if (!mt_pow2_polys[0]) {
        mt_pow2_polys[0] = calloc(MT_PW + 1, sizeof(uint64_t));
        mt_pow2_polys[0][0] = 2; /* x */
    }
    for (int i = 1; i <= b; ++i) {
        if (mt_pow2_polys[i]) continue;
        mt_pow2_polys[i] = malloc((MT_PW + 1) * sizeof(uint64_t));
        memcpy(mt_pow2_polys[i], mt_pow2_polys[i - 1], (MT_PW + 1) * sizeof(uint64_t));
        poly_sqr_mod(mt_pow2_polys[i]);
    }
    return mt_pow2_polys[b];
}

/* Eq. (g_v): Y <- g(A) Y = sum_i a_i A^(i-1) Y, with Y in window form
 * (mt[] = x_t..x_{t+623}, idx = 624).  The window is stepped one word at a
 * time and XOR-accumulated wherever the coefficient is one. */
static void mt_apply_poly(mt_state *s, const uint64_t *g)
{
    uint32_t ring[MT_N], acc[MT_N];
    memcpy(ring, s->mt, sizeof ring);
    memset(acc, 0, sizeof acc);
    int h = 0;
    for (int j = 0; j < MT_DEG; ++j) {
        if ((g[j >> 6] >> (j & 63)) & 1u)
            for (int m = 0; m < MT_N; ++m) acc[m] ^= ring[(h + m) % MT_N];
        ring[h] = mt_recur(ring[h], ring[(h + 1) % MT_N], ring[(h + MT_M) % MT_N]);
        h = (h + 1) % MT_N;
    }
    memcpy(s->mt, acc, sizeof acc);
    s->idx = MT_N;
}

/* Bring a state to window form by consuming the words already twisted, then
 * jump the rest (returns the number of words still to skip via polynomials). */
static void mt_jump(mt_state *s, const uint64_t *e_in)
{
    uint64_t e[NBIG];
    memcpy(e, e_in, sizeof e);
    if (s->idx < MT_N) {
        uint64_t rem = MT_N - s->idx;
        int small = 1;
        for (int w = 1; w < NBIG; ++w) if (e[w]) small = 0;
        if (small && e[0] < rem) { s->idx += (uint32_t)e[0]; return; }
        /* e -= rem */
        uint64_t borrow = rem;
        for (int w = 0; w < NBIG && borrow; ++w) {
            uint64_t before = e[w];
            e[w] -= borrow;
            borrow = (before < borrow) ? 1 : 0;
        }
        s->idx = MT_N;
    }
    /* A^e = prod over set bits b of A^(2^b) (binary decomposition, Sec. 5.4). */
    for (int b = 0; b < 64 * NBIG; ++b)
        if (big_bit(e, b)) mt_apply_poly(s, mt_pow2_poly(b));
}

/* Apply an arbitrary polynomial (used by the period check in the tests). */
void orc_mt_apply_poly(uint32_t *st, const uint64_t *g)
{
    mt_state *s = (mt_state *)st;
    if (s->idx < MT_N) return;         /* window form (idx == 624) only */
    mt_apply_poly(s, g);
}

/* ================================================================== */
/* MRG32K3A (Sec. 5.2)                                                 */
/* ================================================================== */

#define MRG_M1 4294967087ull   /* 2^32 - 209 */
#define MRG_M2 4294944443ull   /* 2^32 - 22853 */

typedef struct { uint64_t x[3]; uint64_t y[3]; } mrg_state; /* (x_n, x_{n-1}, x_{n-2}) */

static const int64_t MRG_A[3][3] = { { 0, 1403580, -810728 }, { 1, 0, 0 }, { 0, 1, 0 } };
static const int64_t MRG_B[3][3] = { { 527612, 0, -1370589 }, { 1, 0, 0 }, { 0, 1, 0 } };

static uint64_t mod_signed(int64_t a, uint64_t m)
{
    int64_t r = a % (int64_t)m;
    return (uint64_t)(r < 0 ? r + (int64_t)m : r);
}

static void mat3_mul(uint64_t r[3][3], uint64_t a[3][3], uint64_t b[3][3], uint64_t m)
{
    uint64_t t[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            u128 acc = 0;
            for (int k = 0; k < 3; ++k) acc += (u128)a[i][k] * b[k][j];
            t[i][j] = (uint64_t)(acc % m);
        }
    memcpy(r, t, sizeof t);
}

static void mat3_vec(uint64_t v[3], uint64_t a[3][3], uint64_t m)
{
    uint64_t t[3];
    for (int i = 0; i < 3; ++i) {
        u128 acc = 0;
        for (int k = 0; k < 3; ++k) acc += (u128)a[i][k] * v[k];
        t[i] = (uint64_t)(acc % m);
    }
    memcpy(v, t, sizeof t);
}

/* r = M^e mod m by square-and-multiply. */
static void mat3_pow(uint64_t r[3][3], const int64_t M[3][3], const uint64_t *e, uint64_t m)
{
    uint64_t base[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { base[i][j] = mod_signed(M[i][j], m); r[i][j] = (i == j); }
    int nb = big_nbits(e);
    for (int b = 0; b < nb; ++b) {
        if (big_bit(e, b)) mat3_mul(r, r, base, m);
        mat3_mul(base, base, base, m);
    }
}

static void mrg_seed(mrg_state *s, uint64_t seed)
{
    if (seed == SEED_DEFAULT) {
        for (int i = 0; i < 3; ++i) s->x[i] = s->y[i] = 12345;
        return;
    }
    uint64_t sm = seed;
    do { for (int i = 0; i < 3; ++i) s->x[i] = splitmix64(&sm) % MRG_M1; } while (!(s->x[0] | s->x[1] | s->x[2]));
    do { for (int i = 0; i < 3; ++i) s->y[i] = splitmix64(&sm) % MRG_M2; } while (!(s->y[0] | s->y[1] | s->y[2]));
}

static uint32_t mrg_next(mrg_state *s)
{
    uint64_t xn = (uint64_t)(((u128)1403580 * s->x[1] + (u128)(MRG_M1 - 810728) * s->x[2]) % MRG_M1);
    uint64_t yn = (uint64_t)(((u128)527612 * s->y[0] + (u128)(MRG_M2 - 1370589) * s->y[2]) % MRG_M2);
    s->x[2] = s->x[1]; s->x[1] = s->x[0]; s->x[0] = xn;
    s->y[2] = s->y[1]; s->y[1] = s->y[0]; s->y[0] = yn;
    uint64_t z = (xn > yn) ? xn - yn : xn + MRG_M1 - yn;   /* (x - y) mod m1, 0 -> m1 */
    return (uint32_t)z;
}

static void mrg_jump(mrg_state *s, const uint64_t *e)
{
    uint64_t a[3][3], b[3][3];
    mat3_pow(a, MRG_A, e, MRG_M1);
    mat3_pow(b, MRG_B, e, MRG_M2);
    mat3_vec(s->x, a, MRG_M1);
    mat3_vec(s->y, b, MRG_M2);
}

/* ================================================================== */
/* LFSR113 (Sec. 5.3)                                                  */
/* ================================================================== */

typedef struct { uint32_t z[4]; } lfsr_state;

static const int LF_P[4] = { 31, 29, 28, 25 };
static const int LF_Q[4] = { 6, 2, 13, 3 };
static const int LF_S[4] = { 18, 2, 7, 13 };

/* One word step of component j: the word holds bits x_{ns}..x_{ns+31}
 * (most significant first, eq. (lfsrOutput)); the top p bits are kept,
 * shifted by s, and the low s bits are refilled through eq. (lfsrRel1). */
static uint32_t lfsr_comp_step(uint32_t z, int j)
{
    int p = LF_P[j], q = LF_Q[j], s = LF_S[j];
    uint32_t mask = 0xFFFFFFFFu << (32 - p);
    uint32_t b = ((z << q) ^ z) >> (p - s);
    return ((z & mask) << s) ^ b;
}

static void lfsr_seed(lfsr_state *st, uint64_t seed)
{
    if (seed == SEED_DEFAULT) { for (int j = 0; j < 4; ++j) st->z[j] = 987654321u; return; }
    uint64_t sm = seed;
    for (int j = 0; j < 4; ++j) {
        uint32_t w;
        do { w = (uint32_t)(splitmix64(&sm) >> 32); } while ((w >> (32 - LF_P[j])) == 0);
        st->z[j] = w;
    }
}

static uint32_t lfsr_next(lfsr_state *st)
{
    uint32_t o = 0;
    for (int j = 0; j < 4; ++j) { st->z[j] = lfsr_comp_step(st->z[j], j); o ^= st->z[j]; }
    return o;
}

/* GF(2) 32x32 matrices as 32 column words: col[i] = image of basis bit i. */
static void gf2_mat_of_step(uint32_t col[32], int j)
{
    for (int i = 0; i < 32; ++i) col[i] = lfsr_comp_step(1u << i, j);
}

static uint32_t gf2_apply(const uint32_t col[32], uint32_t v)
{
    uint32_t r = 0;
    for (int i = 0; i < 32; ++i) if ((v >> i) & 1u) r ^= col[i];
    return r;
}

static void gf2_mul(uint32_t r[32], const uint32_t a[32], const uint32_t b[32]) /* r = a*b */
{
    uint32_t t[32];
    for (int i = 0; i < 32; ++i) t[i] = gf2_apply(a, b[i]);
    memcpy(r, t, sizeof t);
}

static void lfsr_comp_jump(uint32_t *z, int j, const uint64_t *e)
{
    uint32_t base[32], r[32];
    gf2_mat_of_step(base, j);
    for (int i = 0; i < 32; ++i) r[i] = 1u << i;
    int nb = big_nbits(e);
    for (int b = 0; b < nb; ++b) {
        if (big_bit(e, b)) gf2_mul(r, base, r);
        gf2_mul(base, base, base);
    }
    *z = gf2_apply(r, *z);
}

static void lfsr_jump(lfsr_state *st, const uint64_t *e)
{
    for (int j = 0; j < 4; ++j) lfsr_comp_jump(&st->z[j], j, e);
}

/* Bit-level simulation of eq. (lfsrRel1) for one component: given x_0..x_{p-1},
 * produce x_0..x_{nbits-1}. */
void orc_lfsr_bits(int j, const uint8_t *init, uint8_t *x, int nbits)
{
    int p = LF_P[j], q = LF_Q[j];
    for (int i = 0; i < p && i < nbits; ++i) x[i] = init[i];
    for (int n = p; n < nbits; ++n) x[n] = x[n - p] ^ x[n - p + q];
}

/* Component word step, and component jump (for period checks). */
uint32_t orc_lfsr_comp_step(uint32_t z, int j) { return lfsr_comp_step(z, j); }
uint32_t orc_lfsr_comp_jump(uint32_t z, int j, const uint64_t *e) { lfsr_comp_jump(&z, j, e); return z; }
int orc_lfsr_param(int j, int which) { return which == 0 ? LF_P[j] : which == 1 ? LF_Q[j] : LF_S[j]; }

/* ================================================================== */
/* GM / GQ torus-map ensembles (Sec. 5.1, eq. (rec1), Table 2)          */
/* ================================================================== */

typedef struct {
    uint64_t k, q, g;   /* recurrence x' = k x - q x_prev mod g  (Table 2) */
    int v;              /* output bits per point (Table 2)                 */
    int s;              /* points per 32-bit output word (reading, Table 5) */
    int t;              /* g = 2^t p (Sec. 4: "g = p 2^t")                 */
    uint64_t p;
    uint64_t L;         /* block length of the stream-init variant (Table 4) */
    uint64_t nmax;      /* number of sequences of that variant (Table 4)     */
} gm_params_t;

#define GM_MAXPTS 32

typedef struct { uint64_t xp[GM_MAXPTS]; uint64_t xc[GM_MAXPTS]; } gm_state; /* (x^(n-1), x^(n)) */

static int gm_params(int gen, gm_params_t *P)
{
    switch (gen) {
    case O_GM19:   *P = (gm_params_t){ 15, 28, (1ull << 19) - 1, 1, 32, 0, (1ull << 19) - 1, 6000000ull, 1000ull }; return 0;
    case O_GM29:   *P = (gm_params_t){ 4, 2, (1ull << 29) - 3, 1, 32, 0, (1ull << 29) - 3, 80000000ull, 100000000ull }; return 0;
    case O_GM31:   *P = (gm_params_t){ 11, 14, (1ull << 31) - 1, 1, 32, 0, (1ull << 31) - 1, 80000000ull, 1000000000ull }; return 0;
    case O_GM55:   *P = (gm_params_t){ 256, 176, 16ull * ((1ull << 51) - 129), 4, 8, 4, (1ull << 51) - 129, 10000000000ull, 1000000000000000000ull }; return 0;
    case O_GM61:   *P = (gm_params_t){ 24, 74, (1ull << 61) - 1, 1, 32, 0, (1ull << 61) - 1, 10000000000ull, 18000000000000000000ull }; return 0;
    case O_GQ58_1: *P = (gm_params_t){ 8, 48, (1ull << 29) * ((1ull << 29) - 3), 1, 32, 29, (1ull << 29) - 3, 80000000ull, 100000000ull }; return 0;
    case O_GQ58_3: *P = (gm_params_t){ 8, 48, (1ull << 29) * ((1ull << 29) - 3), 3, 12, 29, (1ull << 29) - 3, 80000000ull, 200000000ull }; return 0;
    case O_GQ58_4: *P = (gm_params_t){ 8, 48, (1ull << 29) * ((1ull << 29) - 3), 4, 8, 29, (1ull << 29) - 3, 80000000ull, 300000000ull }; return 0;
    default: return -1;
    }
}

int orc_gm_param(int gen, int which, uint64_t *out)
{
    gm_params_t P;
    if (gm_params(gen, &P)) return -1;
    switch (which) {
    case 0: *out = P.k; break;   case 1: *out = P.q; break;    case 2: *out = P.g; break;
    case 3: *out = (uint64_t)P.v; break; case 4: *out = (uint64_t)P.s; break; case 5: *out = (uint64_t)P.t; break;
    case 6: *out = P.p; break;   case 7: *out = P.L; break;    case 8: *out = P.nmax; break;
    default: return -1;
    }
    return 0;
}

/* eq. (rec1) on one point. */
static uint64_t gm_step1(uint64_t k, uint64_t q, uint64_t g, uint64_t xp, uint64_t xc)
{
    return (uint64_t)(((u128)k * xc + (u128)q * (g - xp)) % g);
}

/* Strip index floor(2^v x / g): which of the 2^v horizontal strips x is in. */
static uint32_t gm_strip(uint64_t x, int v, uint64_t g) { return (uint32_t)(((u128)x << v) / g); }

/* 2x2 matrix M = [[k, -q], [1, 0]] acting on (x^(n), x^(n-1)). */
static void mat2_mul(uint64_t r[4], const uint64_t a[4], const uint64_t b[4], uint64_t g)
{
    uint64_t t[4];
    t[0] = (uint64_t)(((u128)a[0] * b[0] + (u128)a[1] * b[2]) % g);
    t[1] = (uint64_t)(((u128)a[0] * b[1] + (u128)a[1] * b[3]) % g);
    t[2] = (uint64_t)(((u128)a[2] * b[0] + (u128)a[3] * b[2]) % g);
    t[3] = (uint64_t)(((u128)a[2] * b[1] + (u128)a[3] * b[3]) % g);
    memcpy(r, t, sizeof t);
}

/* r = M^e mod g. */
void orc_gm_matpow(uint64_t k, uint64_t q, uint64_t g, const uint64_t *e, uint64_t r[4])
{
    uint64_t base[4] = { k % g, (g - q % g) % g, 1 % g, 0 };
    r[0] = 1 % g; r[1] = 0; r[2] = 0; r[3] = 1 % g;
    int nb = big_nbits(e);
    for (int b = 0; b < nb; ++b) {
        if (big_bit(e, b)) mat2_mul(r, r, base, g);
        mat2_mul(base, base, base, g);
    }
}

static void gm_apply(uint64_t *xp, uint64_t *xc, const uint64_t m[4], uint64_t g)
{
    uint64_t c = (uint64_t)(((u128)m[0] * *xc + (u128)m[1] * *xp) % g);
    uint64_t p = (uint64_t)(((u128)m[2] * *xc + (u128)m[3] * *xp) % g);
    *xc = c; *xp = p;
}

/* Generic single-point helpers (for tests with arbitrary small moduli). */
void orc_gm_point_step(uint64_t k, uint64_t q, uint64_t g, uint64_t *xp, uint64_t *xc)
{
    uint64_t n = gm_step1(k, q, g, *xp, *xc);
    *xp = *xc; *xc = n;
}
void orc_gm_point_jump(uint64_t k, uint64_t q, uint64_t g, uint64_t *xp, uint64_t *xc, const uint64_t *e)
{
    uint64_t m[4];
    orc_gm_matpow(k, q, g, e, m);
    gm_apply(xp, xc, m, g);
}

static void gm_jump(int gen, gm_state *s, const uint64_t *e)
{
    gm_params_t P; gm_params(gen, &P);
    uint64_t m[4];
    orc_gm_matpow(P.k, P.q, P.g, e, m);
    for (int i = 0; i < P.s; ++i) gm_apply(&s->xp[i], &s->xc[i], m, P.g);
}

/* Reading: base pair (x^(0), x^(1)) = 2^t (a, b); (a, b) = (1, 1) for the
 * default seed, else SplitMix64 draws mod p (not both zero).  Point i is the
 * base advanced by i * D, D = nmax * L, so points never overlap below nmax
 * streams (Table 4: s * D <= period). */
/* Table 4: (number of sequences, block length) of the stream-initialisation
 * variants: 0 = the default (init_sequence, or init_short_sequence), 1 =
 * init_medium_sequence, 2 = init_long_sequence.  Block lengths are the printed
 * maximal lengths (GM/GQ) or the powers of two above them (MRG32K3A 2^127,
 * MT19937 2^432, LFSR113 2^34 and 2^80).  Returns -1 for a variant the table
 * does not list. */
int orc_variant(int gen, int v, uint64_t *nmax, uint64_t *L /* NBIG words */)
{
    memset(L, 0, NBIG * sizeof(uint64_t));
    const u128 e7 = 10000000ull, e9 = 1000000000ull, e10 = 10000000000ull;
    u128 l = 0;
    uint64_t nm = 0;
    switch (gen) {
    case O_GM19: if (v == 0) { nm = 1000; l = 6000000; } break;
    case O_GM29: case O_GQ58_1: case O_GQ58_3: case O_GQ58_4: {
        const uint64_t f = gen == O_GQ58_3 ? 2 : gen == O_GQ58_4 ? 3 : 1;
        if (v == 0) { nm = f * 100000000ull; l = 8 * e7; }
        if (v == 1) { nm = f * 1000000ull; l = 8 * e9; }
        if (v == 2) { nm = f * 10000ull; l = 8 * e9 * 100; }
        break;
    }
    case O_GM31:
        if (v == 0) { nm = 1000000000ull; l = 8 * e7; }
        if (v == 1) { nm = 10000000ull; l = 8 * e9; }
        if (v == 2) { nm = 100000ull; l = 8 * e9 * 100; }
        break;
    case O_GM55:
        if (v == 0) { nm = 1000000000000000000ull; l = e10; }
        if (v == 2) { nm = 4000000000ull; l = e10 * e10; }
        break;
    case O_GM61:
        if (v == 0) { nm = 18000000000000000000ull; l = e10; }
        if (v == 2) { nm = 4000000000ull; l = 3 * e10 * e10 * 100000; }
        break;
    case O_LFSR113:
        if (v == 0) { nm = 3800000000000000000ull; l = (u128)1 << 34; }
        if (v == 2) { nm = 4000000000ull; l = (u128)1 << 80; }
        break;
    case O_MRG32K3A: if (v == 0) { nm = 10000000000000000000ull; L[1] = 1ull << 63; if (nmax) *nmax = nm; return 0; } break;
    case O_MT19937: if (v == 0) { nm = 10000000000000000000ull; L[432 / 64] = 1ull << (432 % 64); if (nmax) *nmax = nm; return 0; } break;
    default: break;
    }
    if (!nm) return -1;
    L[0] = (uint64_t)l;
    L[1] = (uint64_t)(l >> 64);
    if (nmax) *nmax = nm;
    return 0;
}

static void gm_seed_v(int gen, int v, gm_state *s, uint64_t seed)
{
    gm_params_t P; gm_params(gen, &P);
    uint64_t a = 1, b = 1;
    if (seed != SEED_DEFAULT) {
        uint64_t sm = seed;
        do { a = splitmix64(&sm) % P.p; b = splitmix64(&sm) % P.p; } while (!(a | b));
    }
    uint64_t x0 = a << P.t, x1 = b << P.t;
    uint64_t D[NBIG] = { 0 }, Lw[NBIG] = { 0 }, nmax = 0;
    orc_variant(gen, v, &nmax, Lw);
    big_mul_u64(D, Lw, nmax);  /* point spacing of the variant's ensemble */
    memset(s, 0, sizeof *s);
    for (int i = 0; i < P.s; ++i) {
        uint64_t e[NBIG];
        big_mul_u64(e, D, (uint64_t)i);
        s->xp[i] = x0; s->xc[i] = x1;
        uint64_t m[4];
        orc_gm_matpow(P.k, P.q, P.g, e, m);
        gm_apply(&s->xp[i], &s->xc[i], m, P.g);
    }
}

static void gm_seed(int gen, gm_state *s, uint64_t seed) { gm_seed_v(gen, 0, s, seed); }

/* Reading of the output: every point takes one step (eq. (rec1)); word =
 * sum_i strip_i << (v*i), truncated to 32 bits, point 0 least significant. */
static uint32_t gm_next(int gen, gm_state *s)
{
    gm_params_t P; gm_params(gen, &P);
    uint64_t word = 0;
    for (int i = 0; i < P.s; ++i) {
        uint64_t n = gm_step1(P.k, P.q, P.g, s->xp[i], s->xc[i]);
        s->xp[i] = s->xc[i]; s->xc[i] = n;
        int sh = P.v * i;
        if (sh < 64) word |= (uint64_t)gm_strip(n, P.v, P.g) << sh;
    }
    return (uint32_t)word;
}

/* ================================================================== */
/* Generic interface used by the tests (gen id, opaque state buffer).   */
/* ================================================================== */

static int is_gm(int gen) { return gen >= O_GM19 && gen <= O_GQ58_4; }

int orc_state_bytes(int gen)
{
    if (gen == O_MT19937) return (int)sizeof(mt_state);
    if (gen == O_MRG32K3A) return (int)sizeof(mrg_state);
    if (gen == O_LFSR113) return (int)sizeof(lfsr_state);
    if (is_gm(gen)) return (int)sizeof(gm_state);
    return -1;
}

int orc_seed(int gen, uint64_t seed, void *st)
{
    if (gen == O_MT19937) { mt_seed(st, seed); return 0; }
    if (gen == O_MRG32K3A) { mrg_seed(st, seed); return 0; }
    if (gen == O_LFSR113) { lfsr_seed(st, seed); return 0; }
    if (is_gm(gen)) { gm_seed(gen, st, seed); return 0; }
    return -1;
}

uint32_t orc_next_u32(int gen, void *st)
{
    if (gen == O_MT19937) return mt_next(st);
    if (gen == O_MRG32K3A) return mrg_next(st);
    if (gen == O_LFSR113) return lfsr_next(st);
    return gm_next(gen, st);
}

int orc_jump(int gen, void *st, const uint64_t *e)
{
    if (gen == O_MT19937) { mt_jump(st, e); return 0; }
    if (gen == O_MRG32K3A) { mrg_jump(st, e); return 0; }
    if (gen == O_LFSR113) { lfsr_jump(st, e); return 0; }
    if (is_gm(gen)) { gm_jump(gen, st, e); return 0; }
    return -1;
}

/* Block length L of the stream-initialisation variant (Table 4; reading:
 * GM/GQ take the printed maximal length, MRG32K3A 2^127 >= 1e38, MT19937
 * 2^432 >= 1e130, LFSR113 2^34 >= 1e10). */
int orc_block_length(int gen, uint64_t *L /* NBIG words */) { return orc_variant(gen, 0, NULL, L); }

/* Stream k of variant v under block splitting: the variant's seeded state
 * (for GM/GQ, the ensemble spaced for that variant) advanced by k * L_v. */
int orc_stream_v(int gen, uint64_t seed, int v, uint64_t k, void *st)
{
    uint64_t L[NBIG], e[NBIG];
    if (orc_variant(gen, v, NULL, L)) return -1;
    if (is_gm(gen)) gm_seed_v(gen, v, st, seed);
    else if (orc_seed(gen, seed, st)) return -1;
    big_mul_u64(e, L, k);
    return orc_jump(gen, st, e);
}

int orc_stream(int gen, uint64_t seed, uint64_t k, void *st) { return orc_stream_v(gen, seed, 0, k, st); }

/* States of streams first..first+n-1 of variant v, laid out back to back:
 * stream first by its own jump, every later one by one more jump of L_v. */
int orc_stream_range_v(int gen, uint64_t seed, int v, uint64_t first, uint64_t n, void *out)
{
    int sb = orc_state_bytes(gen);
    if (sb < 0) return -1;
    uint64_t L[NBIG];
    if (orc_variant(gen, v, NULL, L)) return -1;
    uint8_t *o = out;
    for (uint64_t j = 0; j < n; ++j) {
        if (j == 0) { if (orc_stream_v(gen, seed, v, first, o)) return -1; }
        else { memcpy(o + j * sb, o + (j - 1) * sb, (size_t)sb); orc_jump(gen, o + j * sb, L); }
    }
    return 0;
}

int orc_stream_range(int gen, uint64_t seed, uint64_t first, uint64_t n, void *out)
{
    return orc_stream_range_v(gen, seed, 0, first, n, out);
}

/* Stream k of the spaced layout (Table 3's skip-ahead of 2^sp values): the
 * seeded state of the default variant advanced by k * 2^sp. */
int orc_stream_spaced(int gen, uint64_t seed, uint32_t sp, uint64_t k, void *st)
{
    if (sp + 64 > 64 * NBIG) return -1;
    uint64_t e[NBIG];
    memset(e, 0, sizeof e);
    /* e = k << sp, a 512-bit number */
    const int w = (int)(sp / 64), b = (int)(sp % 64);
    e[w] = k << b;
    if (b && w + 1 < NBIG) e[w + 1] = k >> (64 - b);
    if (is_gm(gen)) gm_seed_v(gen, 0, st, seed);
    else if (orc_seed(gen, seed, st)) return -1;
    return orc_jump(gen, st, e);
}

/* ------------------------------------------------------------------ */
/* Statistical tests (Knuth, TAOCP vol. 2, Sec. 3.3.2): cell counts.   */
/* ------------------------------------------------------------------ */

/* Frequency test: the top b bits of each word select one of 2^b cells. */
void orc_freq_counts(const uint32_t *u, uint64_t n, int b, uint64_t *cnt)
{
    memset(cnt, 0, sizeof(uint64_t) << b);
    for (uint64_t i = 0; i < n; ++i) cnt[u[i] >> (32 - b)] += 1;
}

/* Serial test on non-overlapping pairs (u[2i], u[2i+1]), i < n/2: the cell is
 * (top b bits of u[2i]) * 2^b + (top b bits of u[2i+1]). */
void orc_serial_counts(const uint32_t *u, uint64_t n, int b, uint64_t *cnt)
{
    memset(cnt, 0, sizeof(uint64_t) << (2 * b));
    for (uint64_t i = 0; i + 1 < n; i += 2) {
        const uint64_t a = u[i] >> (32 - b), c = u[i + 1] >> (32 - b);
        cnt[(a << b) | c] += 1;
    }
}

/* Gap test: word u is a hit when lo <= u < hi (hi <= 2^32, so the range may
 * run to the top word).  Walking the words in order,
 * every hit closes a gap whose length r is the number of non-hits since the
 * previous hit (for the first hit: since the start of the sequence).  Gaps of
 * length r < t go to cell r, longer ones to cell t; the non-hits after the
 * last hit close no gap. */
void orc_gap_counts(const uint32_t *u, uint64_t n, uint64_t lo, uint64_t hi, int t, uint64_t *cnt)
{
    memset(cnt, 0, sizeof(uint64_t) * (size_t)(t + 1));
    uint64_t r = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if ((uint64_t)u[i] >= lo && (uint64_t)u[i] < hi) {
            cnt[r < (uint64_t)t ? r : (uint64_t)t] += 1;
            r = 0;
        } else {
            r += 1;
        }
    }
}

void orc_gen_u32(int gen, void *st, uint32_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_next_u32(gen, st);
}

void orc_gen_f32(int gen, void *st, float *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_u32_to_f32(orc_next_u32(gen, st));
}

void orc_gen_f64(int gen, void *st, double *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t u = orc_next_u32(gen, st);
        out[i] = (gen == O_MRG32K3A) ? orc_mrg_to_f64(u) : orc_u32_to_f64(u);
    }
}

/* Many streams at once, stream-major: out[j*n_per + i] = output i of state j.
 * The states (back to back) are advanced in place. */
void orc_gen_many_u32(int gen, void *states, uint64_t nstreams, uint32_t *out, uint64_t n_per)
{
    int sb = orc_state_bytes(gen);
    for (uint64_t j = 0; j < nstreams; ++j) orc_gen_u32(gen, (uint8_t *)states + j * sb, out + j * n_per, n_per);
}
void orc_gen_many_f32(int gen, void *states, uint64_t nstreams, float *out, uint64_t n_per)
{
    int sb = orc_state_bytes(gen);
    for (uint64_t j = 0; j < nstreams; ++j) orc_gen_f32(gen, (uint8_t *)states + j * sb, out + j * n_per, n_per);
}
void orc_gen_many_f64(int gen, void *states, uint64_t nstreams, double *out, uint64_t n_per)
{
    int sb = orc_state_bytes(gen);
    for (uint64_t j = 0; j < nstreams; ++j) orc_gen_f64(gen, (uint8_t *)states + j * sb, out + j * n_per, n_per);
}
