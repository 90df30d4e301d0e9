// stats.cu -- on-device statistics of trajectory ensembles for the
// validation workloads (the paper's Sec. 4 comparisons: two-sample
// Kolmogorov-Smirnov statistic and Wasserstein-1 distance between the
// ensembles of two precision modes; telegraph OFF-state dwell times).
//
// Definitions (integer-exact; the oracle follows the same ones):
//  * count histogram: h[k] = #{v = k}, k = 0..bins-1; values below 0 or
//    above bins-1 go to the end bins and are counted separately;
//  * KS / W1 from two histograms: C_a, C_b cumulative counts, n_a, n_b
//    totals, diff(k) = |C_a(k) n_b - C_b(k) n_a| in 64-bit integers,
//    D = max diff / (n_a n_b), W1 = sum diff / (n_a n_b), each quotient one
//    binary64 division of the two integers (rounded to binary64 first);
//    NaN when a sample is empty or bins n_a n_b >= 2^63;
//  * dwell histogram: per trajectory of a series s[k] (nonzero = OFF),
//    every completed OFF interval, from the first OFF sample after an ON
//    sample to the first ON sample after it: h[end - start] += 1.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ssa.h"

namespace {

constexpr int kSharedBins = 8192;   // privatised block histogram up to this many bins

template <typename T>
__global__ void count_hist_kernel(const T *v, int64_t n, int bins, unsigned long long *hist,
                                  unsigned long long *clamped)
{
    extern __shared__ unsigned int sh[];
    const bool shared = bins <= kSharedBins;
    if (shared)
        for (int k = threadIdx.x; k < bins; k += blockDim.x) sh[k] = 0u;
    __syncthreads();
    unsigned int outside = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)v[i];
        if (x < 0) { x = 0; outside += 1; }
        if (x >= bins) { x = bins - 1; outside += 1; }
        if (shared) atomicAdd(&sh[x], 1u);
        else atomicAdd(&hist[x], 1ull);
    }
    for (int o = 16; o > 0; o >>= 1) outside += __shfl_xor_sync(0xFFFFFFFFu, outside, o);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(clamped, (unsigned long long)outside);
    __syncthreads();
    if (shared)
        for (int k = threadIdx.x; k < bins; k += blockDim.x)
            if (sh[k]) atomicAdd(&hist[k], (unsigned long long)sh[k]);
}

// One block of 1024 threads: thread t owns a contiguous run of bins.
__global__ void __launch_bounds__(1024) ks_w1_kernel(const unsigned long long *ha, const unsigned long long *hb,
                                                     int bins, double *out)
{
    __shared__ long long s_a[1024], s_b[1024];
    __shared__ unsigned long long s_max[1024], s_sum[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (bins + T - 1) / T;
    const int lo = t * chunk < bins ? t * chunk : bins, hi = lo + chunk < bins ? lo + chunk : bins;
    long long la = 0, lb = 0;
    for (int k = lo; k < hi; ++k) {
        la += (long long)ha[k];
        lb += (long long)hb[k];
    }
    s_a[t] = la;
    s_b[t] = lb;
    __syncthreads();
    // inclusive scan of the per-thread totals (Hillis-Steele)
    for (int off = 1; off < T; off <<= 1) {
        const long long va = t >= off ? s_a[t - off] : 0, vb = t >= off ? s_b[t - off] : 0;
        __syncthreads();
        s_a[t] += va;
        s_b[t] += vb;
        __syncthreads();
    }
    const long long na = s_a[T - 1], nb = s_b[T - 1];
    long long ca = t > 0 ? s_a[t - 1] : 0, cb = t > 0 ? s_b[t - 1] : 0;
    unsigned long long dmax = 0, dsum = 0;
    for (int k = lo; k < hi; ++k) {
        ca += (long long)ha[k];
        cb += (long long)hb[k];
        const long long d = ca * nb - cb * na;
        const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
        dmax = ad > dmax ? ad : dmax;
        dsum += ad;
    }
    __syncthreads();
    s_max[t] = dmax;
    s_sum[t] = dsum;
    __syncthreads();
    for (int off = T / 2; off > 0; off >>= 1) {
        if (t < off) {
            s_max[t] = s_max[t] > s_max[t + off] ? s_max[t] : s_max[t + off];
            s_sum[t] += s_sum[t + off];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double nan = __longlong_as_double(0x7FF8000000000000ll);
        if (na <= 0 || nb <= 0 || (double)bins * (double)na * (double)nb >= 9223372036854775808.0) {
            out[0] = nan;
            out[1] = nan;
        } else {
            const double denom = __ll2double_rn(na * nb);
            out[0] = __ull2double_rn(s_max[0]) / denom;
            out[1] = __ull2double_rn(s_sum[0]) / denom;
        }
    }
}

template <typename T>
__global__ void dwell_kernel(const T *s, int K, int64_t n, int64_t k_stride, unsigned long long *hist)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int start = -1;
    bool prev_off = s[j] != 0;
    for (int k = 1; k < K; ++k) {
        const bool off = s[(int64_t)k * k_stride + j] != 0;
        if (off && !prev_off) {
            start = k;
        } else if (!off && prev_off && start >= 0) {
            atomicAdd(&hist[k - start], 1ull);
            start = -1;
        }
        prev_off = off;
    }
}

}  // namespace

extern "C" {

int ssa_count_histogram(const void *values, int elem_bytes, int64_t n, int bins, uint64_t *hist,
                        uint64_t *n_clamped, void *stream)
{
    if (elem_bytes != 2 && elem_bytes != 4) return SSA_EINVAL;
    if (n < 0 || bins < 1 || bins > (1 << 24) || (n > 0 && (!values || !hist || !n_clamped))) return SSA_EINVAL;
    if (n == 0) return SSA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return SSA_ECUDA;
    long long grid = (n + 255) / 256;
    if (grid > (long long)sms * 8) grid = (long long)sms * 8;
    const size_t smem = bins <= kSharedBins ? (size_t)bins * 4 : 0;
    auto *h = reinterpret_cast<unsigned long long *>(hist);
    auto *c = reinterpret_cast<unsigned long long *>(n_clamped);
    if (elem_bytes == 4)
        count_hist_kernel<int32_t><<<(unsigned)grid, 256, smem, s>>>(static_cast<const int32_t *>(values), n, bins, h, c);
    else
        count_hist_kernel<int16_t><<<(unsigned)grid, 256, smem, s>>>(static_cast<const int16_t *>(values), n, bins, h, c);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_hist_ks_w1(const uint64_t *ha, const uint64_t *hb, int bins, double *out, void *stream)
{
    if (!ha || !hb || !out || bins < 1 || bins > (1 << 24)) return SSA_EINVAL;
    ks_w1_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const unsigned long long *>(ha), reinterpret_cast<const unsigned long long *>(hb), bins, out);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_dwell_histogram(const void *series, int elem_bytes, int K, int64_t n, int64_t k_stride, uint64_t *hist,
                        void *stream)
{
    if (elem_bytes != 2 && elem_bytes != 4) return SSA_EINVAL;
    if (K < 1 || n < 0 || k_stride < n || (n > 0 && (!series || !hist))) return SSA_EINVAL;
    if (n == 0) return SSA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)((n + 255) / 256);
    auto *h = reinterpret_cast<unsigned long long *>(hist);
    if (elem_bytes == 4) dwell_kernel<int32_t><<<grid, 256, 0, s>>>(static_cast<const int32_t *>(series), K, n, k_stride, h);
    else dwell_kernel<int16_t><<<grid, 256, 0, s>>>(static_cast<const int16_t *>(series), K, n, k_stride, h);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

}  // extern "C"
