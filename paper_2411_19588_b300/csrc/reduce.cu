// Deterministic column sums of small row-major tables (per-tile and
// per-block partials of the medium gradient, per-block loss partials).
// Stage 1 spreads the rows over kColsumParts CTAs (one row per thread per
// step, coalesced) and reduces each column inside the CTA in a fixed order;
// the caller's final stage adds the kColsumParts partial rows.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace splash {
namespace {

constexpr int kColsumThreads = 256;

// partial row `b` (of kColsumParts) of a table's column sums
template <int COLS>
__device__ __forceinline__ void colsum_part(const float *__restrict__ data, int rows, float *__restrict__ part, int b)
{
    __shared__ float s_w[kColsumThreads / 32][COLS];
    float acc[COLS];
#pragma unroll
    for (int c = 0; c < COLS; c++) acc[c] = 0.f;
    for (int r = b * kColsumThreads + threadIdx.x; r < rows; r += kColsumParts * kColsumThreads)
#pragma unroll
        for (int c = 0; c < COLS; c++) acc[c] += data[(size_t)r * COLS + c];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < COLS; c++) {
        float v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_w[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < COLS) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kColsumThreads / 32; w++) v += s_w[w][threadIdx.x];
        part[b * COLS + threadIdx.x] = v;
    }
}

template <int COLS>
__global__ void __launch_bounds__(kColsumThreads) k_colsum_partial(const float *__restrict__ data, int rows,
                                                                   float *__restrict__ part)
{
    pdl_enter();
    colsum_part<COLS>(data, rows, part, blockIdx.x);
}

// the partial rows of two tables in one launch: CTAs [0, kColsumParts) take
// table a, the next kColsumParts table b
template <int CA, int CB>
__global__ void __launch_bounds__(kColsumThreads) k_colsum_pair(const float *__restrict__ a, int rows_a,
                                                                float *__restrict__ part_a, const float *__restrict__ b,
                                                                int rows_b, float *__restrict__ part_b)
{
    pdl_enter();
    if (blockIdx.x < kColsumParts)
        colsum_part<CA>(a, rows_a, part_a, blockIdx.x);
    else
        colsum_part<CB>(b, rows_b, part_b, blockIdx.x - kColsumParts);
}

}  // namespace

void launch_colsum_pair_6_9(const float *a, int rows_a, float *part_a, const float *b, int rows_b, float *part_b,
                            cudaStream_t s)
{
    launch_pdl(k_colsum_pair<6, 9>, 2 * kColsumParts, kColsumThreads, 0, s, a, rows_a, part_a, b, rows_b, part_b);
    count_launch();
}

void launch_colsum_partial(const float *data, int rows, int cols, float *part, cudaStream_t s)
{
    switch (cols) {
    case 2: launch_pdl(k_colsum_partial<2>, kColsumParts, kColsumThreads, 0, s, data, rows, part); break;
    case 6: launch_pdl(k_colsum_partial<6>, kColsumParts, kColsumThreads, 0, s, data, rows, part); break;
    default: launch_pdl(k_colsum_partial<9>, kColsumParts, kColsumThreads, 0, s, data, rows, part); break;
    }
    count_launch();
}

}  // namespace splash
