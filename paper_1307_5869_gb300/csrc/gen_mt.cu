// MT19937 (Matsumoto & Nishimura 1998; Sec. 5.4): seeding, warp-cooperative
// generation and the polynomial jump-ahead of eq. (g_v).
//
// One warp owns one stream.  The 624-word state lives in shared memory and is
// twisted by the 32 lanes in the three dependency phases of the recurrence
// x_{t+624} = x_{t+397} ^ twist(x_t^u | x_{t+1}^l): words 0..226 read only old
// words, words 227..453 read words 0..226 of the new block, words 454..623 read
// words 227..396 of the new block (Table 5 uses 227 threads per stream for the
// same reason).  Each new word leaves tempered straight from registers, 32
// consecutive words per store instruction.
//
// State layout: stream j at state[j * 624 .. j * 624 + 623].  All streams of a
// handle share the position inside the current block (the handle's index), so
// the index is kept on the host.
//
// Jump (Sec. 5.4): A^v Y = g_v(A) Y = sum_i a_i A^(i-1) Y with g_v = x^v mod phi.
// With Y in window form (x_t..x_{t+623}), A^i Y is the window starting at
// x_{t+i}, so the sum is a sliding-window XOR over the stream's next 20560
// words, taken at the set coefficients of g_v.
#include "mt_dev.cuh"

namespace prand {

constexpr int kMtWarpsPerBlock = 4;

// ------------------------------------------------------------------ seeding
// seed < 2^32: init_genrand(seed); wider seeds: init_by_array({lo32, hi32});
// PRAND_SEED_DEFAULT: init_genrand(5489).  One thread (the recurrence is serial).
__global__ void mt_seed_kernel(uint32_t *base, uint64_t seed)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto genrand_init = [&](uint32_t s) {
        base[0] = s;
        for (uint32_t i = 1; i < kMtN; ++i) base[i] = 1812433253u * (base[i - 1] ^ (base[i - 1] >> 30)) + i;
    };
    if (seed == PRAND_SEED_DEFAULT) { genrand_init(5489u); return; }
    if (seed <= 0xFFFFFFFFull) { genrand_init((uint32_t)seed); return; }
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    genrand_init(19650218u);
    int i = 1, j = 0;
    for (int k = kMtN; k; --k) {
        base[i] = (base[i] ^ ((base[i - 1] ^ (base[i - 1] >> 30)) * 1664525u)) + key[j] + (uint32_t)j;
        ++i; ++j;
        if (i >= kMtN) { base[0] = base[kMtN - 1]; i = 1; }
        if (j >= 2) j = 0;
    }
    for (int k = kMtN - 1; k; --k) {
        base[i] = (base[i] ^ ((base[i - 1] ^ (base[i - 1] >> 30)) * 1566083941u)) - (uint32_t)i;
        ++i;
        if (i >= kMtN) { base[0] = base[kMtN - 1]; i = 1; }
    }
    base[0] = 0x80000000u;
}

// ------------------------------------------------------------------ generation
template <typename OutT>
__global__ void __launch_bounds__(32 * kMtWarpsPerBlock) mt_gen_kernel(uint32_t *state, uint64_t nstreams, uint32_t idx0,
                                                                       uint64_t nper, OutT *__restrict__ out)
{
    __shared__ uint32_t sm[kMtWarpsPerBlock][2][kMtN];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t j = (uint64_t)blockIdx.x * kMtWarpsPerBlock + w;
    if (j >= nstreams) return;  // whole warp
    uint32_t *b0 = sm[w][0], *b1 = sm[w][1];
    const uint32_t *src = state + j * kMtN;
    mt_copy_state_warp(src, b0, lane);
    __syncwarp();
    OutT *o = out + j * nper;
    uint64_t done = 0;
    // the rest of the current block
    if (idx0 < (uint32_t)kMtN) {
        const uint32_t cnt = (uint32_t)min((uint64_t)(kMtN - idx0), nper);
        for (uint32_t t = lane; t < cnt; t += 32) o[t] = Cvt<OutT>::f(mt_temper(b0[idx0 + t]));
        done = cnt;
    }
    // whole new blocks, each twisted once and emitted as it is made; the loop
    // is unrolled by two so both calls see fixed shared-memory buffers
    bool in_b0 = true;
    while (done < nper) {
        uint64_t rem = nper - done;
        uint32_t emit = rem < (uint64_t)kMtN ? (uint32_t)rem : (uint32_t)kMtN;
        mt_twist_emit<OutT>(b0, b1, lane, o + done, emit);
        done += emit;
        in_b0 = false;
        if (done >= nper) break;
        rem = nper - done;
        emit = rem < (uint64_t)kMtN ? (uint32_t)rem : (uint32_t)kMtN;
        mt_twist_emit<OutT>(b1, b0, lane, o + done, emit);
        done += emit;
        in_b0 = true;
    }
    const uint32_t *cur = in_b0 ? b0 : b1;
    uint32_t *dst = state + j * kMtN;
    mt_copy_state_warp(cur, dst, lane);
}

// ------------------------------------------------------------------ jump
// Doubling level: dst stream (off + j) := g(A) (src stream j), j < count.
__global__ void __launch_bounds__(32 * kMtWarpsPerBlock) mt_level_kernel(const uint32_t *poly, uint32_t *state,
                                                                         uint64_t off, uint64_t count)
{
    __shared__ uint32_t seq[kMtWarpsPerBlock][2 * kMtN], pbuf[kMtWarpsPerBlock][kMtPolyWords];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t j = (uint64_t)blockIdx.x * kMtWarpsPerBlock + w;
    if (j >= count) return;
    mt_apply_poly_warp(poly, state + j * kMtN, state + (off + j) * kMtN, seq[w], pbuf[w], lane);
}

// Every stream advanced by the set bits of a 512-bit offset (one polynomial
// x^(2^b) mod phi per set bit b, applied one after another in place).
struct MtBits { uint64_t w[8]; };

__global__ void __launch_bounds__(32 * kMtWarpsPerBlock) mt_multi_kernel(const uint32_t *polys, uint32_t *state,
                                                                         uint64_t n, MtBits e, uint32_t *scratch)
{
    __shared__ uint32_t seq[kMtWarpsPerBlock][2 * kMtN], pbuf[kMtWarpsPerBlock][kMtPolyWords];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t j = (uint64_t)blockIdx.x * kMtWarpsPerBlock + w;
    if (j >= n) return;
    uint32_t *s = state + j * kMtN;
    for (int b = 0; b < 512; ++b) {
        if (!((e.w[b >> 6] >> (b & 63)) & 1u)) continue;
        // result goes to registers then back over s (src is copied to smem first)
        mt_apply_poly_warp(polys + (size_t)b * kMtPolyWords, s, s, seq[w], pbuf[w], lane);
        __syncwarp();
    }
    (void)scratch;
}

// ------------------------------------------------------------------ host
static unsigned grid_warps(uint64_t n) { return (unsigned)((n + kMtWarpsPerBlock - 1) / kMtWarpsPerBlock); }

prand_status_t mt_seed(uint64_t seed, void *d_base, cudaStream_t st)
{
    mt_seed_kernel<<<1, 32, 0, st>>>((uint32_t *)d_base, seed);
    return launch_check();
}

// streams j = 0..n-1 := base advanced by (first + j) * 2^shift (2^432 in the
// Table 4 layout): stream 0 by the bits of first, then a doubling tree
// (stream 2^b + j from stream j by 2^(shift + b)).
prand_status_t mt_init(const DevTables *T, const void *d_base, void *d_state, uint64_t first, uint64_t n, cudaStream_t st,
                       int shift)
{
    uint32_t *state = (uint32_t *)d_state;
    if (cudaMemcpyAsync(state, d_base, kMtN * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return PRAND_ERR_CUDA;
    if (first) {
        MtBits e = {};
        // first * 2^shift: bits shift .. shift + 63
        for (int b = 0; b < 64; ++b)
            if ((first >> b) & 1u) e.w[(shift + b) >> 6] |= 1ull << ((shift + b) & 63);
        mt_multi_kernel<<<1, 32 * kMtWarpsPerBlock, 0, st>>>(T->mt, state, 1, e, nullptr);
        prand_status_t s = launch_check();
        if (s != PRAND_OK) return s;
    }
    for (int b = 0; b < 64 && (1ull << b) < n; ++b) {
        uint64_t have = 1ull << b;
        uint64_t count = min(have, n - have);
        mt_level_kernel<<<grid_warps(count), 32 * kMtWarpsPerBlock, 0, st>>>(
            T->mt + (size_t)(shift + b) * kMtPolyWords, state, have, count);
        prand_status_t s = launch_check();
        if (s != PRAND_OK) return s;
    }
    return PRAND_OK;
}

// Skip ahead: consume the rest of the current block, then jump by polynomials.
// Every stream += off (512 bits, off < 2^512 as for the paper's a 2^b form):
// the rest of the current block is used up by moving the index, the remainder
// is one polynomial x^(2^b) mod phi per set bit.
prand_status_t mt_skip512(const DevTables *T, void *d_state, uint64_t n, uint32_t *idx, const uint64_t off_in[8],
                          cudaStream_t st)
{
    MtBits e = {};
    for (int i = 0; i < 8; ++i) e.w[i] = off_in[i];
    if (*idx < (uint32_t)kMtN) {
        uint64_t rem = kMtN - *idx;
        bool small = true;
        for (int i = 1; i < 8; ++i) small = small && !e.w[i];
        if (small && e.w[0] < rem) { *idx += (uint32_t)e.w[0]; return PRAND_OK; }
        uint64_t borrow = rem;
        for (int i = 0; i < 8 && borrow; ++i) {
            uint64_t before = e.w[i];
            e.w[i] -= borrow;
            borrow = before < borrow ? 1 : 0;
        }
        *idx = kMtN;
    }
    bool any = false;
    for (int i = 0; i < 8; ++i) any = any || e.w[i];
    if (!any) return PRAND_OK;
    mt_multi_kernel<<<grid_warps(n), 32 * kMtWarpsPerBlock, 0, st>>>(T->mt, (uint32_t *)d_state, n, e, nullptr);
    return launch_check();
}

prand_status_t mt_skip(const DevTables *T, void *d_state, uint64_t n, uint32_t *idx, const U256 &off, cudaStream_t st)
{
    const uint64_t w[8] = { off.w[0], off.w[1], off.w[2], off.w[3], 0, 0, 0, 0 };
    return mt_skip512(T, d_state, n, idx, w, st);
}

prand_status_t mt_gen(void *d_state, uint64_t nstreams, uint32_t *idx, void *out, int dtype, uint64_t nper, cudaStream_t st)
{
    uint32_t *state = (uint32_t *)d_state;
    unsigned grid = grid_warps(nstreams);
    if (dtype == PRAND_DTYPE_U32) mt_gen_kernel<uint32_t><<<grid, 32 * kMtWarpsPerBlock, 0, st>>>(state, nstreams, *idx, nper, (uint32_t *)out);
    else if (dtype == PRAND_DTYPE_F32) mt_gen_kernel<float><<<grid, 32 * kMtWarpsPerBlock, 0, st>>>(state, nstreams, *idx, nper, (float *)out);
    else mt_gen_kernel<double><<<grid, 32 * kMtWarpsPerBlock, 0, st>>>(state, nstreams, *idx, nper, (double *)out);
    prand_status_t s = launch_check();
    if (s != PRAND_OK) return s;
    // the index after nper outputs: the rest of the current block, then whole blocks
    uint64_t avail = kMtN - *idx;
    if (nper <= avail) *idx += (uint32_t)nper;
    else *idx = (uint32_t)((nper - avail - 1) % kMtN + 1);
    return PRAND_OK;
}

}  // namespace prand
