// ssa_order.cu -- the ordering step of longest-first scheduling.
//
// Between the two launches of the direct-method kernel, the parked
// trajectories are put in descending order of their predicted remaining work
// a0(x) * (t_end - t), evaluated here in binary32 from the parked state and
// the run's rate constants (a priority only), so that launch 2 starts the long
// ones first and ends on short ones: a persistent queue then finishes close to
// the mean load of its lanes instead of waiting for a long trajectory that
// happened to start last.  The order is a counting sort over 1024 buckets of
// the key (16 per octave); items within a bucket land in any order.  Results
// never depend on it: every trajectory's random numbers are keyed by its id
// and event count.
#include <cuda_runtime.h>

#include <cstdint>

#include "ssa_launch.h"

namespace ssa {

namespace {

constexpr int kBuckets = kOrderBuckets;

// Monotone in key >= 0: the exponent and top four mantissa bits of key + 1.
__device__ __forceinline__ int key_bucket(float key)
{
    const int b = (__float_as_int(key + 1.0f) >> 19) - (127 << 4);
    return min(max(b, 0), kBuckets - 1);
}

// Bucket of item i, or -1 when it was not parked.
__device__ __forceinline__ int item_bucket(const OrderModel &m, int64_t i, int64_t n)
{
    if (!m.parked[i]) return -1;
    const int64_t set = m.n_sets > 1 ? i / m.traj_per_set : 0;
    float a0 = 0.0f;
#pragma unroll 1
    for (int j = 0; j < m.M; ++j) {
        float v;
        if (m.law[j] == 1) {
            const float xr = (float)m.x[(int64_t)m.hill_reg[j] * n + i];
            float q = 1.0f;
            for (int r = 0; r < m.hill_h[j]; ++r) q *= xr;
            const bool tab = m.n_sets > 1 && m.hill_tab;
            const float h0 = tab ? (float)m.hill_tab[(set * m.M + j) * 2 + 0] : m.h0[j];
            const float h1 = tab ? (float)m.hill_tab[(set * m.M + j) * 2 + 1] : m.h1[j];
            v = h0 + h1 / (1.0f + q);
        } else {
            v = m.n_sets > 1 ? (float)m.cprime_tab[set * m.M + j] : m.c[j];
#pragma unroll 1
            for (int s = 0; s < m.N; ++s) {
                if (m.folded[j][s]) continue;
                const int x = m.x[(int64_t)s * n + i];
                for (int r = 0; r < m.order[j][s]; ++r) v *= (float)max(x - r, 0);
            }
        }
        a0 += v;
    }
    const float key = a0 * (float)(m.t_end - m.t[i]);
    return key == key ? key_bucket(fmaxf(key, 0.0f)) : 0;
}

__global__ void __launch_bounds__(256) order_count_kernel(const OrderModel m, int64_t n, unsigned *hist)
{
    __shared__ unsigned h[kBuckets];
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int b = item_bucket(m, i, n);
        if (b >= 0) atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One block of kBuckets threads: offs[b] = entries in the buckets above b
// (largest keys first), *count = all entries.
__global__ void __launch_bounds__(kBuckets) order_offsets_kernel(const unsigned *hist, unsigned long long *offs,
                                                                  unsigned long long *count)
{
    __shared__ unsigned long long s[kBuckets];
    const int t = threadIdx.x;
    const int b = kBuckets - 1 - t;   // position t holds bucket b: descending keys
    const unsigned long long own = hist[b];
    s[t] = own;
    __syncthreads();
    for (int d = 1; d < kBuckets; d <<= 1) {
        const unsigned long long v = t >= d ? s[t - d] : 0ull;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    offs[b] = s[t] - own;
    if (t == kBuckets - 1) *count = s[t];
}

// Scatter with one atomic per bucket and warp (lanes of a warp that share a
// bucket reserve their slots together).
__global__ void __launch_bounds__(256) order_scatter_kernel(const OrderModel m, int64_t n, unsigned long long *offs,
                                                            int64_t *order)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    // warp-uniform trip count: every lane of the warp takes part in each round
    for (int64_t w = first; w < n; w += stride) {
        const int64_t i = w + lane;
        const int b = i < n ? item_bucket(m, i, n) : -1;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
        const int leader = __ffs(peers) - 1;
        unsigned long long base = 0ull;
        if (b >= 0 && (int)lane == leader) base = atomicAdd(&offs[b], (unsigned long long)__popc(peers));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (b >= 0) order[base + (unsigned long long)__popc(peers & ((1u << lane) - 1u))] = i;
    }
}

}  // namespace

cudaError_t launch_order(const OrderModel &m, int64_t n, unsigned *hist, unsigned long long *offs,
                         unsigned long long *count, int64_t *order, cudaStream_t stream, int *launches)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * kBuckets, stream);
    if (e != cudaSuccess) return e;
    long long grid = (n + 255) / 256;
    if (grid > (long long)sms * 8) grid = (long long)sms * 8;
    if (grid < 1) grid = 1;
    order_count_kernel<<<(unsigned)grid, 256, 0, stream>>>(m, n, hist);
    order_offsets_kernel<<<1, kBuckets, 0, stream>>>(hist, offs, count);
    order_scatter_kernel<<<(unsigned)grid, 256, 0, stream>>>(m, n, offs, order);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace ssa
