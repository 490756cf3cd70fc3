// The float maps (Sec. 7.3: outputs uniform in [0, 1)) applied to a caller's
// array of 32-bit outputs, with the same device functions the generators use
// for their f32 / f64 epilogue.
#include <algorithm>

#include "devcommon.cuh"

namespace prand {
namespace {

template <typename OutT, bool MRG, bool VEC>
__global__ void __launch_bounds__(256) convert_kernel(const uint32_t *__restrict__ in, uint64_t n, OutT *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (VEC) {
        // four outputs per thread and iteration: one 16-byte load, 16- or 32-byte stores
        const uint64_t n4 = n / 4;
        for (uint64_t q = t0; q < n4; q += stride) {
            const uint4 u = reinterpret_cast<const uint4 *>(in)[q];
            store4<OutT>(out + 4 * q, Cvt<OutT, MRG>::f(u.x), Cvt<OutT, MRG>::f(u.y), Cvt<OutT, MRG>::f(u.z),
                         Cvt<OutT, MRG>::f(u.w));
        }
        for (uint64_t i = 4 * n4 + t0; i < n; i += stride) out[i] = Cvt<OutT, MRG>::f(in[i]);
    } else {
        for (uint64_t i = t0; i < n; i += stride) out[i] = Cvt<OutT, MRG>::f(in[i]);
    }
}

template <typename OutT, bool MRG>
prand_status_t launch(const uint32_t *in, uint64_t n, void *out, cudaStream_t st)
{
    const int sms = device_sm_count();
    const uint64_t want = (n / 4 + 255) / 256;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 8));
    const bool vec = (uintptr_t)in % 16 == 0 && (uintptr_t)out % (sizeof(OutT) == 8 ? 32 : 16) == 0;
    if (vec) convert_kernel<OutT, MRG, true><<<grid, 256, 0, st>>>(in, n, (OutT *)out);
    else convert_kernel<OutT, MRG, false><<<grid, 256, 0, st>>>(in, n, (OutT *)out);
    return launch_check();
}

}  // namespace
}  // namespace prand

using namespace prand;

extern "C" prand_status_t prand_convert(const uint32_t *dev_in, uint64_t n, int32_t map, void *dev_out,
                                        prand_stream_t stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    if ((!dev_in || !dev_out) && n) return PRAND_ERR_ARG;
    if (map != PRAND_DTYPE_F32 && map != PRAND_DTYPE_F64 && map != PRAND_MAP_MRG_F64) return PRAND_ERR_ARG;
    if (n == 0) return PRAND_OK;
    const size_t es = map == PRAND_DTYPE_F32 ? 4 : 8;
    if ((uintptr_t)dev_in % 4 != 0 || (uintptr_t)dev_out % es != 0) return PRAND_ERR_ALIGN;
    if (map == PRAND_DTYPE_F32) return launch<float, false>(dev_in, n, dev_out, stream);
    if (map == PRAND_DTYPE_F64) return launch<double, false>(dev_in, n, dev_out, stream);
    return launch<double, true>(dev_in, n, dev_out, stream);
}
