// Statistical tests of generated words: the frequency, serial and gap tests of
// Knuth (TAOCP vol. 2, Sec. 3.3.2), in the role TestU01 plays in the paper's
// study of the generators and of their skip-ahead subsequences (Secs. 3-4,
// Tables 1 and 3).  The GPU computes the cell counts (one pass over the words,
// bound by reading them from HBM); the host turns counts into Pearson's
// statistic and its chi-square tail probability.
#include <algorithm>
#include <cmath>

#include "devcommon.cuh"

namespace prand {
namespace {

constexpr unsigned kBlock = 256;
constexpr int kGapChunkLog = 13;  // words per gap chunk (one warp each)
constexpr uint32_t kMaxGapT = 1024;
constexpr unsigned kStitchThreads = 1024;

bool test_valid(const prand_test_t *t)
{
    if (!t) return false;
    switch (t->kind) {
    case PRAND_TEST_FREQUENCY: return t->bits >= 1 && t->bits <= 12;
    case PRAND_TEST_SERIAL: return t->bits >= 1 && t->bits <= 6;
    case PRAND_TEST_GAP: return t->lo < t->hi && t->hi <= (1ull << 32) && t->t >= 1 && t->t <= kMaxGapT;
    default: return false;
    }
}

uint32_t cells_of(const prand_test_t *t)
{
    if (!test_valid(t)) return 0;
    if (t->kind == PRAND_TEST_FREQUENCY) return 1u << t->bits;
    if (t->kind == PRAND_TEST_SERIAL) return 1u << (2 * t->bits);
    return t->t + 1;
}

// ------------------------------------------------------------ frequency, serial
// Each block counts into shared memory (reps copies of the cells, one per
// group of warps, so few cells do not serialise every atomic on one word),
// then adds its non-zero cells to the global counts.  Grid-stride over
// 16-byte vectors when the words are 16-byte aligned.
template <bool SERIAL, bool VEC>
__global__ void __launch_bounds__(kBlock) hist_kernel(const uint32_t *__restrict__ u, uint64_t n, uint32_t bits,
                                                      uint32_t cells, uint32_t reps,
                                                      unsigned long long *__restrict__ counts)
{
    extern __shared__ uint32_t h[];
    for (uint32_t i = threadIdx.x; i < reps * cells; i += blockDim.x) h[i] = 0;
    __syncthreads();
    uint32_t *my = h + ((threadIdx.x >> 5) % reps) * cells;
    const uint32_t sh = 32 - bits;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!SERIAL) {
        uint64_t i0 = 0;
        if (VEC) {
            const uint64_t n4 = n / 4;
            for (uint64_t q = t0; q < n4; q += stride) {
                const uint4 v = reinterpret_cast<const uint4 *>(u)[q];
                atomicAdd(&my[v.x >> sh], 1u);
                atomicAdd(&my[v.y >> sh], 1u);
                atomicAdd(&my[v.z >> sh], 1u);
                atomicAdd(&my[v.w >> sh], 1u);
            }
            i0 = 4 * n4;
        }
        for (uint64_t i = i0 + t0; i < n; i += stride) atomicAdd(&my[u[i] >> sh], 1u);
    } else {
        // pair p = (u[2p], u[2p+1]), p < n / 2
        const uint64_t np = n / 2;
        uint64_t p0 = 0;
        if (VEC) {
            const uint64_t n4 = n / 4;  // two pairs per vector
            for (uint64_t q = t0; q < n4; q += stride) {
                const uint4 v = reinterpret_cast<const uint4 *>(u)[q];
                atomicAdd(&my[((v.x >> sh) << bits) | (v.y >> sh)], 1u);
                atomicAdd(&my[((v.z >> sh) << bits) | (v.w >> sh)], 1u);
            }
            p0 = 2 * n4;
        }
        for (uint64_t p = p0 + t0; p < np; p += stride)
            atomicAdd(&my[((u[2 * p] >> sh) << bits) | (u[2 * p + 1] >> sh)], 1u);
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) {
        uint32_t s = 0;
        for (uint32_t r = 0; r < reps; ++r) s += h[r * cells + c];
        if (s) atomicAdd(&counts[c], (unsigned long long)s);
    }
}

// ------------------------------------------------------------------ gap
// One warp per chunk of 2^13 words, read 32 consecutive words per round (one
// per lane).  The round's hits form a ballot mask in sequence order, so a
// hit's predecessor is the highest set bit below its lane, or the last hit of
// an earlier round.  Positions inside a chunk are 32-bit offsets, kept as
// offset + 1 so that 0 means "no hit yet"; a gap is (offset of the hit) -
// (offset of the previous hit + 1).  The hit test is one unsigned compare:
// u - lo <= hi - lo - 1.  The first hit of a chunk needs the previous chunk's
// last hit, so it is left to the stitch kernel: each chunk records its first
// and last hit (absolute position + 1; 0 = no hit).
// Shared-memory cells of a block: cells 0..t of the gap lengths, then one
// dummy cell per lane.  Every lane adds 1 in every step -- to its gap's cell
// when it closes a gap, else to its own dummy cell -- so the increment needs
// neither a branch nor a predicate, and the dummies never collide.
__device__ __forceinline__ void red_shared(uint32_t addr)
{
    asm volatile("red.shared.add.u32 [%0], 1;" :: "r"(addr));
}

template <bool FULL>
__device__ __forceinline__ void gap_chunk(const uint32_t *__restrict__ u, uint32_t len, uint32_t lo, uint32_t span_m1,
                                          uint32_t t, uint32_t hs, int lane, uint32_t &first1, uint32_t &prev1)
{
    constexpr int U = 8;  // rounds whose loads are issued together
    const unsigned below_mask = (1u << lane) - 1u;
    const uint32_t dummy = hs + 4u * (t + 1 + lane);
    for (uint32_t r0 = 0; r0 < len; r0 += 32 * U) {
        uint32_t x[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t i = r0 + 32 * k + lane;
            x[k] = (FULL || i < len) ? u[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t r = r0 + 32 * k;
            const bool hit = (FULL || r + lane < len) && x[k] - lo <= span_m1;
            const unsigned m = __ballot_sync(kFull, hit);
            const unsigned below = m & below_mask;
            const uint32_t p1 = below ? r + 32 - __clz(below) : prev1;
            red_shared((hit && p1) ? hs + 4u * min(r + lane - p1, t) : dummy);
            if (!prev1 && m) first1 = r + __ffs(m);  // warp-uniform: once per chunk
            prev1 = m ? r + 32 - __clz(m) : prev1;
        }
    }
}

// The same for a whole chunk of 16-byte aligned words, four consecutive words
// per lane and round (128 words): a lane's hits are walked in order, starting
// from the last hit before its words -- the last hit of the nearest lower lane
// that has one (ballot of "lane has a hit", one shuffle), or of an earlier
// round.  One ballot per 128 words instead of one per 32.
__device__ __forceinline__ void gap_chunk_vec(const uint32_t *__restrict__ u, uint32_t lo, uint32_t span_m1,
                                              uint32_t t, uint32_t hs, int lane, uint32_t &first1, uint32_t &prev1)
{
    constexpr uint32_t C = 1u << kGapChunkLog;
    constexpr int U = 4;  // rounds whose loads are issued together
    const unsigned below_mask = (1u << lane) - 1u;
    const uint32_t dummy = hs + 4u * (t + 1 + lane);
    for (uint32_t r0 = 0; r0 < C; r0 += 128 * U) {
        uint4 v[U];
#pragma unroll
        for (int k = 0; k < U; ++k) v[k] = *reinterpret_cast<const uint4 *>(u + r0 + 128 * k + 4 * lane);
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t b = r0 + 128 * k + 4 * lane;  // offset of this lane's first word
            const bool h0 = v[k].x - lo <= span_m1, h1 = v[k].y - lo <= span_m1;
            const bool h2 = v[k].z - lo <= span_m1, h3 = v[k].w - lo <= span_m1;
            const uint32_t last = h3 ? b + 4 : h2 ? b + 3 : h1 ? b + 2 : h0 ? b + 1 : 0u;
            const unsigned lm = __ballot_sync(kFull, last != 0u);
            const unsigned below = lm & below_mask;
            const uint32_t from = __shfl_sync(kFull, last, below ? 31 - __clz(below) : lane);
            if (!prev1 && lm) {  // warp-uniform: the chunk's first hit, once per chunk
                const uint32_t firsthere = h0 ? b + 1 : h1 ? b + 2 : h2 ? b + 3 : b + 4;
                first1 = __shfl_sync(kFull, firsthere, __ffs(lm) - 1);
            }
            uint32_t p1 = below ? from : prev1;
#define PRAND_GAP_WORD(H, J)                                                   \
            red_shared(((H) && p1) ? hs + 4u * min(b + (J) - p1, t) : dummy);  \
            p1 = (H) ? b + (J) + 1 : p1;
            PRAND_GAP_WORD(h0, 0)
            PRAND_GAP_WORD(h1, 1)
            PRAND_GAP_WORD(h2, 2)
            PRAND_GAP_WORD(h3, 3)
#undef PRAND_GAP_WORD
            prev1 = lm ? __reduce_max_sync(kFull, last) : prev1;
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kBlock) gap_chunk_kernel(const uint32_t *__restrict__ u, uint64_t n, uint32_t lo,
                                                           uint32_t span_m1, uint32_t t, uint64_t nchunks,
                                                           unsigned long long *__restrict__ counts,
                                                           unsigned long long *__restrict__ first1,
                                                           unsigned long long *__restrict__ last1)
{
    __shared__ uint32_t h[kMaxGapT + 1 + 32];  // cells 0..t, then the lanes' dummy cells
    for (uint32_t i = threadIdx.x; i <= t + 32; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t hs = (uint32_t)__cvta_generic_to_shared(h);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    constexpr uint32_t C = 1u << kGapChunkLog;
    for (uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; c < nchunks; c += nwarps) {
        const uint64_t base = c << kGapChunkLog;
        const uint32_t len = (uint32_t)min((uint64_t)C, n - base);
        uint32_t f1 = 0, p1 = 0;
        if (len == C) {
            if (VEC) gap_chunk_vec(u + base, lo, span_m1, t, hs, lane, f1, p1);
            else gap_chunk<true>(u + base, C, lo, span_m1, t, hs, lane, f1, p1);
        } else {
            gap_chunk<false>(u + base, len, lo, span_m1, t, hs, lane, f1, p1);
        }
        if (lane == 0) {
            first1[c] = f1 ? base + f1 : 0ull;
            last1[c] = p1 ? base + p1 : 0ull;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i <= t; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], (unsigned long long)h[i]);
}

// Gaps that end at the first hit of a chunk.  Thread k walks a contiguous run
// of chunks and counts the gaps whose previous hit lies in its run; the gap
// before its run's first hit takes the last hit of all earlier runs (a max
// scan over the runs' last hits, since positions grow with the run index; 0
// stands for the start of the sequence, i.e. a virtual hit at position -1).
__global__ void __launch_bounds__(kStitchThreads) gap_stitch_kernel(const unsigned long long *__restrict__ first1,
                                                                    const unsigned long long *__restrict__ last1,
                                                                    uint64_t nchunks, uint32_t t,
                                                                    unsigned long long *__restrict__ counts)
{
    __shared__ unsigned long long scan[kStitchThreads];
    __shared__ uint32_t h[kMaxGapT + 1];
    for (uint32_t i = threadIdx.x; i <= t; i += blockDim.x) h[i] = 0;
    const uint64_t per = (nchunks + kStitchThreads - 1) / kStitchThreads;
    const uint64_t c0 = min((uint64_t)threadIdx.x * per, nchunks), c1 = min(c0 + per, nchunks);
    __syncthreads();
    uint64_t mine = 0, prev = 0;  // this run's first hit, its latest hit (position + 1; 0 = none)
    constexpr int B = 8;          // records loaded together
    for (uint64_t cb = c0; cb < c1; cb += B) {
        uint64_t f[B], l[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            f[k] = cb + k < c1 ? first1[cb + k] : 0ull;
            l[k] = cb + k < c1 ? last1[cb + k] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (!f[k]) continue;
            if (prev) {
                const uint64_t g = f[k] - prev - 1;
                atomicAdd(&h[g < t ? (uint32_t)g : t], 1u);
            } else {
                mine = f[k];
            }
            prev = l[k];
        }
    }
    scan[threadIdx.x] = prev;
    __syncthreads();
    for (unsigned d = 1; d < kStitchThreads; d <<= 1) {
        const unsigned long long v = threadIdx.x >= d ? scan[threadIdx.x - d] : 0ull;
        __syncthreads();
        if (v > scan[threadIdx.x]) scan[threadIdx.x] = v;
        __syncthreads();
    }
    if (mine) {
        const uint64_t before = threadIdx.x ? scan[threadIdx.x - 1] : 0ull;
        const uint64_t g = mine - before - 1;
        atomicAdd(&h[g < t ? (uint32_t)g : t], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i <= t; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], (unsigned long long)h[i]);
}

unsigned grid_for_words(uint64_t units)
{
    const int sms = device_sm_count();
    const uint64_t want = (units + kBlock - 1) / kBlock;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 8));
}

// ------------------------------------------------------------------ host math
// Q(a, x) = Gamma(a, x) / Gamma(a), the regularized upper incomplete gamma
// function: below x = a + 1 as 1 - P(a, x) with P's power series
//   P(a, x) = e^-x x^a / Gamma(a + 1) * sum_n x^n / ((a + 1) ... (a + n)),
// above it by the continued fraction
//   Gamma(a, x) = e^-x x^a / (x + 1 - a - 1 (1 - a) / (x + 3 - a - 2 (2 - a) / (x + 5 - a - ...)))
// evaluated with the modified Lentz method (Lentz 1976; Thompson & Barnett 1986).
double gamma_q(double a, double x)
{
    if (x <= 0.0) return 1.0;
    const double lead = std::exp(-x + a * std::log(x) - std::lgamma(a));
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term;
        for (int k = 1; k < 100000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (std::fabs(term) <= std::fabs(sum) * 1e-17) break;
        }
        return std::max(0.0, 1.0 - lead * sum);
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, f = d;
    for (int k = 1; k < 100000; ++k) {
        const double an = -k * (k - a);
        b += 2.0;
        d = an * d + b;
        if (std::fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        f *= del;
        if (std::fabs(del - 1.0) <= 1e-16) break;
    }
    return lead * f;
}

}  // namespace
}  // namespace prand

using namespace prand;

extern "C" {

uint32_t prand_test_cells(const prand_test_t *test) { return cells_of(test); }

prand_status_t prand_test_counts(const prand_test_t *test, const uint32_t *dev_words, uint64_t n,
                                 uint64_t *dev_counts, prand_stream_t stream)
{
    const uint32_t cells = cells_of(test);
    if (!cells || !dev_counts || (!dev_words && n) || n >= (1ull << 40)) return PRAND_ERR_ARG;
    if ((uintptr_t)dev_words % 4 || (uintptr_t)dev_counts % 8) return PRAND_ERR_ALIGN;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(dev_counts, 0, (size_t)cells * sizeof(uint64_t), st) != cudaSuccess) return PRAND_ERR_CUDA;
    if (n == 0) return PRAND_OK;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(dev_counts);
    if (test->kind != PRAND_TEST_GAP) {
        const bool serial = test->kind == PRAND_TEST_SERIAL;
        const uint32_t reps = std::max<uint32_t>(1, std::min<uint32_t>(8, 4096 / cells));
        const size_t smem = (size_t)reps * cells * sizeof(uint32_t);
        const bool vec = (uintptr_t)dev_words % 16 == 0;
        const unsigned grid = grid_for_words(vec ? n / 4 : n);
        if (serial) {
            if (vec) hist_kernel<true, true><<<grid, kBlock, smem, st>>>(dev_words, n, test->bits, cells, reps, cnt);
            else hist_kernel<true, false><<<grid, kBlock, smem, st>>>(dev_words, n, test->bits, cells, reps, cnt);
        } else {
            if (vec) hist_kernel<false, true><<<grid, kBlock, smem, st>>>(dev_words, n, test->bits, cells, reps, cnt);
            else hist_kernel<false, false><<<grid, kBlock, smem, st>>>(dev_words, n, test->bits, cells, reps, cnt);
        }
        return launch_check();
    }
    const uint64_t nchunks = (n + (1ull << kGapChunkLog) - 1) >> kGapChunkLog;
    unsigned long long *rec = nullptr;
    if (cudaMallocAsync((void **)&rec, (size_t)nchunks * 2 * sizeof(unsigned long long), st) != cudaSuccess) {
        cudaGetLastError();
        return PRAND_ERR_NOMEM;
    }
    const unsigned grid = grid_for_words(nchunks * 32);
    const uint32_t lo = (uint32_t)test->lo, span_m1 = (uint32_t)(test->hi - test->lo - 1);
    if ((uintptr_t)dev_words % 16 == 0)
        gap_chunk_kernel<true><<<grid, kBlock, 0, st>>>(dev_words, n, lo, span_m1, test->t, nchunks, cnt, rec,
                                                        rec + nchunks);
    else
        gap_chunk_kernel<false><<<grid, kBlock, 0, st>>>(dev_words, n, lo, span_m1, test->t, nchunks, cnt, rec,
                                                         rec + nchunks);
    prand_status_t s = launch_check();
    if (s == PRAND_OK) {
        gap_stitch_kernel<<<1, kStitchThreads, 0, st>>>(rec, rec + nchunks, nchunks, test->t, cnt);
        s = launch_check();
    }
    if (cudaFreeAsync(rec, st) != cudaSuccess && s == PRAND_OK) s = PRAND_ERR_CUDA;
    return s;
}

double prand_chi2_sf(double x, double dof)
{
    if (!(x >= 0.0) || !(dof > 0.0) || std::isinf(dof)) return std::nan("");
    if (std::isinf(x)) return 0.0;
    return gamma_q(0.5 * dof, 0.5 * x);
}

prand_status_t prand_test_evaluate(const prand_test_t *test, uint64_t n, const uint64_t *host_counts, double *chi2,
                                   double *dof, double *pvalue)
{
    const uint32_t cells = cells_of(test);
    if (!cells || !host_counts) return PRAND_ERR_ARG;
    double e_flat = 0.0, G = 0.0, p = 0.0;
    if (test->kind == PRAND_TEST_FREQUENCY) {
        e_flat = (double)n / cells;
    } else if (test->kind == PRAND_TEST_SERIAL) {
        e_flat = (double)(n / 2) / cells;
    } else {
        for (uint32_t i = 0; i < cells; ++i) G += (double)host_counts[i];
        p = (double)(test->hi - test->lo) / 4294967296.0;
    }
    double stat = 0.0;
    for (uint32_t i = 0; i < cells; ++i) {
        double e = e_flat;
        if (test->kind == PRAND_TEST_GAP)
            e = i < test->t ? G * p * std::pow(1.0 - p, (double)i) : G * std::pow(1.0 - p, (double)test->t);
        if (!(e > 0.0)) return PRAND_ERR_ARG;
        const double d = (double)host_counts[i] - e;
        stat += d * d / e;
    }
    const double k = (double)(cells - 1);
    if (chi2) *chi2 = stat;
    if (dof) *dof = k;
    if (pvalue) *pvalue = prand_chi2_sf(stat, k);
    return PRAND_OK;
}

}  // extern "C"
