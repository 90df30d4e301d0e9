// mlp_tc.cu -- tcgen05 GEMM with fused epilogues, pack kernels, and the GEMM
// test entry of the C ABI.  See mlp_tc.cuh for the operand layout.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/ssa.h"
#include "mlp_tc.cuh"

namespace mlp {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between core matrices along K), stride byte offset (between 8-row
// groups along M/N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 32 lanes x 16 consecutive fp32 columns: thread t of the warp gets its row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t f2bf(float x)
{
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    return cdf + z * pdf;
}

// 16 bf16 values of row r, columns c0..c0+15 into a packed matrix with C columns
__device__ __forceinline__ void store_packed16(uint8_t *base, int64_t r, int c0, int C, const uint16_t (&h)[16])
{
    uint4 lo, hi;
    lo.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    lo.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
    lo.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
    lo.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
    hi.x = (uint32_t)h[8] | ((uint32_t)h[9] << 16);
    hi.y = (uint32_t)h[10] | ((uint32_t)h[11] << 16);
    hi.z = (uint32_t)h[12] | ((uint32_t)h[13] << 16);
    hi.w = (uint32_t)h[14] | ((uint32_t)h[15] << 16);
    *reinterpret_cast<uint4 *>(base + packed_offset(r, c0, C)) = lo;
    *reinterpret_cast<uint4 *>(base + packed_offset(r, c0 + 8, C)) = hi;
}

// ------------------------------------------------------------ the GEMM
__global__ void __launch_bounds__(128, 1) gemm_kernel(const __grid_constant__ GemmArgs g)
{
    extern __shared__ uint8_t dyn_smem[];
    __shared__ uint64_t bars[4];          // operands landed in stage 0 / 1, MMAs reading stage 0 / 1 done
    __shared__ uint32_t tmem_base_s;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dyn_smem) + 127) & ~uintptr_t(127));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int nt = g.ntile, n0 = blockIdx.y * nt;     // this CTA's columns n0 .. n0 + nt - 1
    const uint32_t ncols = nt <= 32 ? 32u : (nt <= 64 ? 64u : (nt <= 128 ? 128u : 256u));
    if (warp == 0) tmem_alloc(&tmem_base_s, ncols);
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = tmem_base_s;

    const int n_chunks = g.K / g.kchunk;
    const uint32_t idesc = instr_desc_bf16_f32(kTileM, nt);
    const uint32_t rg_bytes = (uint32_t)g.kchunk * 16u;   // one 8-row group of one stage
    const uint32_t stage_bytes = (uint32_t)(kTileM + nt) * (uint32_t)g.kchunk * 2u;
    const uint32_t limit = g.spin_limit ? g.spin_limit : kSpinLimit;

    // With two stages (g.stages, set when the reduction has several chunks and
    // both fit in shared memory) the copies of chunk c + 1 land while the MMAs
    // of chunk c run.  Stage c % stages holds chunk c; its barriers complete
    // once per use, so chunk c waits for parity (c / stages) & 1.
    const int stages = g.stages == 2 ? 2 : 1;
    auto stage_a = [&](int st) { return smem + (size_t)st * stage_bytes; };
    auto issue_load = [&](int c) {   // warp 0, all lanes
        const int st = c % stages;
        uint8_t *sA = stage_a(st), *sB = sA + (size_t)kTileM * g.kchunk * 2;
        if (lane == 0) mbar_expect_tx(&bars[st], stage_bytes);
        __syncwarp();
        const int colA = g.a_col0 + c * g.kchunk, colB = g.b_col0 + c * g.kchunk;
        const int groups = kTileM / 8 + nt / 8;
        for (int q = lane; q < groups; q += 32) {
            if (q < kTileM / 8) {
                const int64_t rg = (int64_t)tile * (kTileM / 8) + q;
                bulk_g2s(sA + (size_t)q * rg_bytes, g.A + (rg * (g.lda_cols / 8) + colA / 8) * 128, rg_bytes,
                         &bars[st]);
            } else {
                const int64_t rg = q - kTileM / 8;
                const int64_t brg = (int64_t)(n0 / 8) + rg;
                bulk_g2s(sB + (size_t)rg * rg_bytes, g.B + (brg * (g.ldb_cols / 8) + colB / 8) * 128, rg_bytes,
                         &bars[st]);
            }
        }
    };
    // issued work whose completion has not been observed (the same in every
    // thread): the chunk loading into each stage, the last chunk committed
    int pend_load[2] = {-1, -1};
    int pend_mma = -1;
    int err = ERR_NONE;
    for (int c = 0; c < stages && c < n_chunks; ++c) {
        if (warp == 0 && g.withhold != 1) issue_load(c);
        if (g.withhold != 1) pend_load[c] = c;
    }
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int st = ch % stages;
        const uint32_t parity = (uint32_t)((ch / stages) & 1);
        if (!__syncthreads_and(mbar_wait(&bars[st], parity, limit))) {
            err = ERR_LOAD_TIMEOUT;
            break;
        }
        pend_load[st] = -1;
        tc_fence_after();
        if (tid == 0 && g.withhold != 2) {
            const uint32_t a0 = smem_addr(stage_a(st)), b0 = a0 + (uint32_t)kTileM * (uint32_t)g.kchunk * 2u;
            for (int s = 0; s < g.kchunk / 16; ++s) {
                const uint64_t ad = smem_desc(a0 + (uint32_t)s * 256u, 128u, rg_bytes);
                const uint64_t bd = smem_desc(b0 + (uint32_t)s * 256u, 128u, rg_bytes);
                mma_bf16(tmem_d, ad, bd, idesc, (ch > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(&bars[2 + st]);   // arrives once every MMA issued so far has completed
        }
        if (g.withhold != 2) pend_mma = ch;
        __syncwarp();
        // stage st is reused by chunk ch + stages once these MMAs have read
        // it; the last chunk's MMAs must be complete before the epilogue
        if (ch + stages < n_chunks || ch == n_chunks - 1) {
            if (!__syncthreads_and(mbar_wait(&bars[2 + st], parity, limit))) {
                err = ERR_MMA_TIMEOUT;
                break;
            }
            pend_mma = -1;   // commits are cumulative: every earlier MMA is done too
            if (ch + stages < n_chunks) {
                if (warp == 0 && g.withhold != 1) issue_load(ch + stages);
                if (g.withhold != 1) pend_load[st] = ch + stages;
            }
        }
    }
    const bool ok = err == ERR_NONE;   // the same in every thread
    tc_fence_after();

    if (ok) {
        const int64_t row = (int64_t)tile * kTileM + warp * 32 + lane;
        const bool valid = row < g.m_valid;
        for (int cl = 0; cl < nt; cl += 16) {
            const int c0 = n0 + cl;       // column of D
            float v[16];
            tmem_ld16(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)cl, v);
            if (g.epi == EPI_STORE_F32 || g.epi == EPI_LOGITS) {
                if (valid) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        g.fout[row * g.ld_fout + c0 + i] = v[i] + (g.epi == EPI_LOGITS ? g.bias[c0 + i] : 0.0f);
                }
            } else {
                uint16_t h[16];
                float dz[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float y;
                    if (g.epi == EPI_HIDDEN_FWD) {
                        const float z = v[i] + g.bias[c0 + i];
                        if (valid) g.fout[row * g.ld_fout + c0 + i] = z;
                        y = gelu(z);
                    } else {
                        y = valid ? v[i] * gelu_grad(g.zin[row * g.N + c0 + i]) : 0.0f;
                    }
                    if (!valid) y = 0.0f;
                    dz[i] = y;
                    h[i] = f2bf(y);
                }
                store_packed16(g.pk_out, row, c0, g.N, h);
                if (g.pkT_out) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        *reinterpret_cast<uint16_t *>(g.pkT_out + packed_offset(c0 + i, row, g.pkT_cols)) = h[i];
                }
                if (g.epi == EPI_HIDDEN_BWD && g.bias_grad) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float s = dz[i];
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                        if (lane == 0) atomicAdd(&g.bias_grad[c0 + i], s);
                    }
                }
            }
        }
    } else {
        if (tid == 0) atomicExch(g.error, err);
        // let our own copies and MMAs still in flight land (bounded) before the
        // CTA frees its tensor memory and leaves its shared memory
        for (int st = 0; st < stages; ++st)
            if (pend_load[st] >= 0) mbar_wait(&bars[st], (uint32_t)((pend_load[st] / stages) & 1), kSpinLimit);
        if (pend_mma >= 0)
            mbar_wait(&bars[2 + pend_mma % stages], (uint32_t)((pend_mma / stages) & 1), kSpinLimit);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem_d, ncols);
}

// ------------------------------------------------------------ packing
// Row-major bf16 [rows][cols] (leading dimension ld) -> packed [rows_pad][C].
// One thread per 16-byte core-matrix row; padding is zero.
__global__ void pack_bf16_kernel(const uint16_t *src, int rows, int cols, int ld, uint8_t *dst, int rows_pad, int C)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_row = C / 8;
    if (idx >= (int64_t)rows_pad * per_row) return;
    const int64_t r = idx / per_row;
    const int c0 = (int)(idx % per_row) * 8;
    uint16_t h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = (r < rows && c0 + i < cols) ? src[r * ld + c0 + i] : (uint16_t)0;
    uint4 v;
    v.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    v.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
    v.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
    v.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
    *reinterpret_cast<uint4 *>(dst + packed_offset(r, c0, C)) = v;
}

namespace {
int g_withhold = 0;
uint32_t g_spin_limit = 0;
}  // namespace

void set_wait_test(int withhold, uint32_t spin_limit)
{
    g_withhold = withhold;
    g_spin_limit = spin_limit;
}

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t s)
{
    // Shared memory also caps how many CTAs share an SM: request enough that
    // their tensor-memory columns (ncols each) never exceed the SM's 512.
    GemmArgs a = g;
    a.withhold = g_withhold;
    a.spin_limit = g_spin_limit;
    a.ntile = (g.N >= 128 && g.N % 64 == 0) ? 64 : g.N;   // column tiles per row tile: N / ntile
    const int ncols = a.ntile <= 32 ? 32 : (a.ntile <= 64 ? 64 : (a.ntile <= 128 ? 128 : 256));
    const size_t per_sm = 233472, reserve = 1024;
    const size_t cap_ctas = (size_t)(512 / ncols);
    const size_t stage = (size_t)(kTileM + a.ntile) * (size_t)g.kchunk * 2;
    const size_t max_dyn = 232448;   // 227 KB of dynamic shared memory per CTA
    a.stages = (g.K / g.kchunk > 1 && 2 * stage + 128 <= max_dyn) ? 2 : 1;   // pipeline over several chunks
    size_t smem = (size_t)a.stages * stage + 128;
    const size_t floor_bytes = per_sm / (cap_ctas + 1) + 1 - reserve;
    if (smem < floor_bytes) smem = floor_bytes;
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = (g.M + kTileM - 1) / kTileM;
    const dim3 grid((unsigned)tiles, (unsigned)(g.N / a.ntile));
    gemm_kernel<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

// Packed bf16 [rows_pad][C] -> row-major [rows][C] (one thread per element).
__global__ void unpack_bf16_kernel(const uint8_t *src, int rows, int C, uint16_t *dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * C) return;
    const int64_t r = i / C;
    const int c = (int)(i % C);
    dst[i] = *reinterpret_cast<const uint16_t *>(src + packed_offset(r, c, C));
}

cudaError_t launch_pack(const uint16_t *src, int rows, int cols, int ld, uint8_t *dst, int rows_pad, int C,
                        cudaStream_t s)
{
    const int64_t n = (int64_t)rows_pad * (C / 8);
    pack_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, rows, cols, ld, dst, rows_pad, C);
    return cudaGetLastError();
}

}  // namespace mlp

// ------------------------------------------------------------ C ABI test entries
extern "C" int ssa_mlp_set_wait_test(int withhold, int spin_limit)
{
    if (withhold < 0 || withhold > 2 || spin_limit < 0) return SSA_EINVAL;
    mlp::set_wait_test(withhold, (uint32_t)spin_limit);
    return SSA_OK;
}

extern "C" int ssa_mlp_gemm_epi(int epi, int M, int N, int K, const uint16_t *A, const uint16_t *B,
                                const float *bias, const float *zin, float *fout, uint16_t *hout, float *bias_grad,
                                void *stream)
{
    if (epi < mlp::EPI_STORE_F32 || epi > mlp::EPI_HIDDEN_BWD) return SSA_EINVAL;
    if (M < 1 || N < 16 || N > mlp::kMaxN || N % 16 != 0 || K < 16 || K % 16 != 0 || (K > 256 && K % 256 != 0) ||
        !A || !B)
        return SSA_EINVAL;
    const bool need_f = epi != mlp::EPI_HIDDEN_BWD, need_h = epi == mlp::EPI_HIDDEN_FWD || epi == mlp::EPI_HIDDEN_BWD;
    if ((need_f && !fout) || (need_h && !hout)) return SSA_EINVAL;
    if ((epi == mlp::EPI_HIDDEN_FWD || epi == mlp::EPI_LOGITS) && !bias) return SSA_EINVAL;
    if (epi == mlp::EPI_HIDDEN_BWD && (!zin || !bias_grad)) return SSA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int Mpad = (M + mlp::kTileM - 1) / mlp::kTileM * mlp::kTileM;
    const size_t a_bytes = (size_t)Mpad * K * 2, b_bytes = (size_t)N * K * 2;
    const size_t h_bytes = need_h ? (size_t)Mpad * N * 2 : 0;
    uint8_t *buf = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&buf), a_bytes + b_bytes + h_bytes + 256, s) != cudaSuccess)
        return SSA_ENOMEM;
    int *err = reinterpret_cast<int *>(buf + a_bytes + b_bytes + h_bytes);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = mlp::launch_pack(A, M, K, K, buf, Mpad, K, s);
    if (e == cudaSuccess) e = mlp::launch_pack(B, N, K, K, buf + a_bytes, N, K, s);
    mlp::GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = buf;
    g.B = buf + a_bytes;
    g.lda_cols = K;
    g.ldb_cols = K;
    g.M = M;
    g.m_valid = M;
    g.N = N;
    g.K = K;
    g.kchunk = K > 256 ? 256 : K;
    g.epi = epi;
    g.bias = bias;
    g.zin = zin;
    g.fout = fout;
    g.ld_fout = N;
    g.pk_out = need_h ? buf + a_bytes + b_bytes : nullptr;
    g.bias_grad = bias_grad;
    g.error = err;
    if (e == cudaSuccess) e = mlp::launch_gemm(g, s);
    if (e == cudaSuccess && need_h) {
        const int64_t n = (int64_t)M * N;
        mlp::unpack_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.pk_out, M, N, hout);
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return SSA_ECUDA;
    return herr ? SSA_ETIMEDOUT : SSA_OK;
}

extern "C" int ssa_mlp_gemm_bf16(int M, int N, int K, const uint16_t *A, const uint16_t *B, float *D, void *stream)
{
    if (!D) return SSA_EINVAL;
    return ssa_mlp_gemm_epi(mlp::EPI_STORE_F32, M, N, K, A, B, nullptr, nullptr, D, nullptr, nullptr, stream);
}
