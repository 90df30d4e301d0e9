// round16.cu -- the 16-bit rounding step of the engine, exposed on arrays.
//
// Every reduced-precision operation of the direct method, tau-leaping and
// the RDME ends in one rounding of a binary32 value to binary16 or bfloat16
// (round to nearest even, or stochastic rounding, Sec. 3.3).  This entry
// point applies exactly the device functions the kernels use (rn16 / sr16 of
// ssa_device.cuh, i.e. cvt.rn and cvt.rs) to caller arrays, so the rounding
// contract can be checked in isolation: all random values for a given x,
// subnormal results, the overflow edge, signs and exact values.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ssa.h"
#include "ssa_device.cuh"

namespace {

template <int FMT>
__global__ void round16_kernel(const float *x, const uint32_t *rbits, int64_t n, int rounding, int half, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    out[i] = rounding ? ssa::sr16<FMT>(v, rbits[i], half != 0) : ssa::rn16<FMT>(v);
}

}  // namespace

extern "C" int ssa_round16(const float *x, const uint32_t *rbits, int64_t n, int format, int rounding, int half,
                           float *out, void *stream)
{
    if (n < 0 || (format != 0 && format != 1) || (rounding != 0 && rounding != 1) || (half != 0 && half != 1))
        return SSA_EINVAL;
    if (n == 0) return SSA_OK;
    if (!x || !out || (rounding && !rbits)) return SSA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (format == 0) round16_kernel<0><<<grid, 256, 0, s>>>(x, rbits, n, rounding, half, out);
    else round16_kernel<1><<<grid, 256, 0, s>>>(x, rbits, n, rounding, half, out);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}
