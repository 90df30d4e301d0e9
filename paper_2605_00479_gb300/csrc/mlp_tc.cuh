// mlp_tc.cuh -- tcgen05 (5th-generation tensor core) GEMM for the surrogate MLP.
//
// D[M x N] (fp32, in tensor memory) = sum over K of A[M x K] * B[N x K]^T with
// A and B in bf16.  One CTA of 128 threads owns a 128-row x ntile-column tile
// of D (ntile = 64 when N >= 128 is a multiple of 64, else N; grid = row
// tiles x column tiles); the accumulator occupies ntile columns of tensor
// memory.
//
// Operands live in global memory in the "packed" layout that tcgen05 reads
// without swizzling (K-major core matrices of 8 rows x 16 bytes):
//   byte(r, c) = ((r / 8) * (C / 8) + c / 8) * 128 + (r % 8) * 16 + (c % 8) * 2
// for a matrix with C columns (the reduction dimension).  Producers (the
// epilogues and the pack kernels) write this layout directly, so each stage
// of a GEMM is a few 1-D bulk copies (cp.async.bulk, the TMA's linear mode)
// completing on an mbarrier; one elected thread then issues the MMAs and
// commits them to a second mbarrier (with two stages when the reduction spans
// several chunks, so one chunk's copies land while the previous chunk's MMAs
// run); four warps read the accumulator with
// tcgen05.ld and run a fused epilogue.  Every wait is bounded: on timeout the
// kernel records an error code, waits (bounded) for its own work in flight,
// frees its tensor memory and returns.  Whether a wait ran out is decided for
// the whole CTA at once (__syncthreads_and), so all threads leave together.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mlp {

constexpr int kTileM = 128;
constexpr int kMaxN = 256;
constexpr int kMaxChunk = 256;       // reduction columns per stage
constexpr uint32_t kSpinLimit = 1u << 22;

enum Epilogue {
    EPI_STORE_F32 = 0,     // fout[r][c] = acc
    EPI_HIDDEN_FWD = 1,    // z = acc + bias; fout = z; y = gelu(z) -> packed out (+ transposed)
    EPI_LOGITS = 2,        // fout = acc + bias
    EPI_HIDDEN_BWD = 3,    // dz = acc * gelu'(zin) -> packed out (+ transposed); bias_grad += dz
};

enum ErrorCode { ERR_NONE = 0, ERR_LOAD_TIMEOUT = 1, ERR_MMA_TIMEOUT = 2 };

struct GemmArgs {
    const uint8_t *A;          // packed, rows = M (padded to 128), C = lda_cols
    const uint8_t *B;          // packed, rows = N, C = ldb_cols
    int lda_cols, ldb_cols;    // C of the packed A / B matrices
    int a_col0, b_col0;        // first reduction column used (multiple of 16)
    int M, N, K, kchunk;       // rows of D computed (tiles of 128), columns, reduction length, columns per stage
    int ntile;                 // columns of D per CTA (set by launch_gemm)
    int m_valid;               // rows < m_valid are real; the others are written as zeros (or skipped)
    int epi;
    const float *bias;         // [N]
    const float *zin;          // [M][N] pre-activations (EPI_HIDDEN_BWD)
    float *fout;               // [M][ld_fout]
    int ld_fout;
    uint8_t *pk_out;           // packed bf16 [Mpad][N] (C = N)
    uint8_t *pkT_out;          // packed bf16 [N][MpadT] (C = pkT_cols)
    int pkT_cols;
    float *bias_grad;          // [N], accumulated with atomics
    int *error;                // device error word (0 = ok)
    uint32_t spin_limit;       // polls per bounded wait (0: kSpinLimit)
    int withhold;              // failure-detection test: 1 no operand loads, 2 no MMAs (their waits run out)
    int stages;                // shared-memory stages (1 or 2; set by launch_gemm)
};

// Failure-detection test setting applied by launch_gemm to every later GEMM
// (withhold 0 and spin_limit 0: normal operation).
void set_wait_test(int withhold, uint32_t spin_limit);

__host__ __device__ constexpr uint32_t instr_desc_bf16_f32(int M, int N)
{
    return (1u << 4)                       // D format: f32
           | (1u << 7)                     // A format: bf16
           | (1u << 10)                    // B format: bf16
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__host__ __device__ inline int64_t packed_offset(int64_t r, int64_t c, int64_t C)
{
    return ((r >> 3) * (C >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2;
}

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t s);
__global__ void unpack_bf16_kernel(const uint8_t *src, int rows, int C, uint16_t *dst);
cudaError_t launch_pack(const uint16_t *src, int rows, int cols, int ld, uint8_t *dst, int rows_pad, int C,
                        cudaStream_t s);

}  // namespace mlp
