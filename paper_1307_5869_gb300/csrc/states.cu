// Export / import of a handle's stream states in the one-struct-per-stream
// layout of prand_device.h (the paper's single-threaded state, Sec. 7.3).
#include "prand_internal.h"
#include "prand_device.h"

namespace prand {
namespace {

constexpr unsigned kB = 256;

// one thread per (stream, 32-bit word of the struct)
__global__ void export_mt(const uint32_t *state, uint64_t n, uint32_t idx, uint32_t *out)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * (kMtN + 1)) return;
    const uint64_t j = t / (kMtN + 1), w = t % (kMtN + 1);
    out[t] = w < (uint64_t)kMtN ? state[j * kMtN + w] : idx;
}
__global__ void import_mt(const uint32_t *in, uint64_t n, uint32_t *state)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * kMtN) return;
    const uint64_t j = t / kMtN, w = t % kMtN;
    state[t] = in[j * (kMtN + 1) + w];
}
// every struct's index must equal the first one's (the handle keeps one index)
__global__ void check_mt_idx(const uint32_t *in, uint64_t n, uint32_t *bad)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t v = in[j * (kMtN + 1) + kMtN];
    if (v != in[kMtN] || v > (uint32_t)kMtN) atomicOr(bad, 1u);
}

// word c of stream j: state[c * n + j] <-> struct word j * W + c
template <int W>
__global__ void export_soa(const uint32_t *state, uint64_t n, uint32_t *out)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    const uint64_t j = t / W, c = t % W;
    out[t] = state[c * n + j];
}
template <int W>
__global__ void import_soa(const uint32_t *in, uint64_t n, uint32_t *state)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    const uint64_t j = t / W, c = t % W;
    state[c * n + j] = in[t];
}

// GM: xp[j s + i], xc[(n + j) s + i] <-> struct (x_prev[32], x[32]) of stream j
__global__ void export_gm(const uint64_t *state, uint64_t n, int s, uint64_t *out)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 64) return;
    const uint64_t j = t / 64;
    const int e = (int)(t % 64), i = e & 31;
    out[t] = i < s ? (e < 32 ? state[j * s + i] : state[(n + j) * s + i]) : 0ull;
}
__global__ void import_gm(const uint64_t *in, uint64_t n, int s, uint64_t *state)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 2 * (uint64_t)s) return;
    const uint64_t j = t / (2 * s);
    const int e = (int)(t % (2 * s)), half = e / s, i = e % s;
    state[(half ? n + j : j) * s + i] = in[j * 64 + (half ? 32 : 0) + i];
}

unsigned grid(uint64_t threads) { return (unsigned)((threads + kB - 1) / kB); }

}  // namespace

uint64_t device_state_bytes(int gen)
{
    if (gen == PRAND_MT19937) return sizeof(prand_mt19937_state);
    if (gen == PRAND_MRG32K3A) return sizeof(prand_mrg32k3a_state);
    if (gen == PRAND_LFSR113) return sizeof(prand_lfsr113_state);
    if (is_gm(gen)) return sizeof(prand_gm_state);
    return 0;
}

prand_status_t export_states_dev(int gen, const void *d_state, uint64_t n, uint32_t mt_idx, void *out, cudaStream_t st)
{
    if (gen == PRAND_MT19937)
        export_mt<<<grid(n * (kMtN + 1)), kB, 0, st>>>((const uint32_t *)d_state, n, mt_idx, (uint32_t *)out);
    else if (gen == PRAND_MRG32K3A)
        export_soa<6><<<grid(n * 6), kB, 0, st>>>((const uint32_t *)d_state, n, (uint32_t *)out);
    else if (gen == PRAND_LFSR113)
        export_soa<4><<<grid(n * 4), kB, 0, st>>>((const uint32_t *)d_state, n, (uint32_t *)out);
    else
        export_gm<<<grid(n * 64), kB, 0, st>>>((const uint64_t *)d_state, n, gm_params(gen).s, (uint64_t *)out);
    return launch_check();
}

prand_status_t import_states_dev(int gen, const void *in, uint64_t n, void *d_state, uint32_t *mt_idx, cudaStream_t st)
{
    prand_status_t s;
    if (gen == PRAND_MT19937) {
        uint32_t *bad = nullptr, h_bad = 0, idx = 0;
        if (!dev_alloc(&bad, sizeof(uint32_t))) return PRAND_ERR_NOMEM;
        cudaMemsetAsync(bad, 0, sizeof(uint32_t), st);
        check_mt_idx<<<grid(n), kB, 0, st>>>((const uint32_t *)in, n, bad);
        s = launch_check();
        if (s == PRAND_OK &&
            (cudaMemcpyAsync(&h_bad, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(&idx, (const uint32_t *)in + kMtN, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            s = PRAND_ERR_CUDA;
        cudaFree(bad);
        if (s != PRAND_OK) return s;
        if (h_bad) return PRAND_ERR_STATE;
        import_mt<<<grid(n * kMtN), kB, 0, st>>>((const uint32_t *)in, n, (uint32_t *)d_state);
        if ((s = launch_check()) != PRAND_OK) return s;
        *mt_idx = idx;
        return PRAND_OK;
    }
    if (gen == PRAND_MRG32K3A)
        import_soa<6><<<grid(n * 6), kB, 0, st>>>((const uint32_t *)in, n, (uint32_t *)d_state);
    else if (gen == PRAND_LFSR113)
        import_soa<4><<<grid(n * 4), kB, 0, st>>>((const uint32_t *)in, n, (uint32_t *)d_state);
    else {
        const int sp = gm_params(gen).s;
        import_gm<<<grid(n * 2 * sp), kB, 0, st>>>((const uint64_t *)in, n, sp, (uint64_t *)d_state);
    }
    return launch_check();
}

}  // namespace prand
