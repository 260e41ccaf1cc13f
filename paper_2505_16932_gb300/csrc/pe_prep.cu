// Step S1 of the online stage (Alg. 1 online box; App. A online code):
//   nu = ||G||_F,  X_0 = G / (scale * nu + eps),
// in one pass over G. Each block takes one 64 x 256 strip of the canonical
// short-side layout (X = G^T when m > n), padded with zeros to whole tiles,
// and writes it unscaled in every precision the chosen path needs (FP32;
// BF16 hi with the code of the next 8 bits; BF16 hi + lo), together with the tile's
// sum of squares. The last block to finish (atomic ticket)
// sums each matrix's tile partials in a fixed order and stores the matrix's
// normalisation factor 1 / (scale * nu + eps); the first polynomial step
// applies it (A = s^2 X X^T, X_1 = s (a X + B X)), which is the same map as
// scaling X_0 first.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "pe_internal.h"
#include "pe_prep_body.cuh"

namespace pe {

namespace {

// Three blocks per SM without the momentum path (80 registers; the loads
// of three blocks in flight), two with it (its extra loads need the registers).
template <bool MUON>
__global__ void __launch_bounds__(256, MUON ? 2 : 3) prepare_kernel(const DevMat* __restrict__ mats, int nmats,
                                                      const TileTask* __restrict__ tiles,
                                                      double* __restrict__ partials, float scale, float eps,
                                                      int outputs, float* __restrict__ nscale,
                                                      int* __restrict__ status, int* __restrict__ counters,
                                                      int ncounters, unsigned* __restrict__ ticket) {
    __shared__ float tile[64][65];
    __shared__ double red[8];
    __shared__ int s_last;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < ncounters; i += blockDim.x) counters[i] = 0;
    }
    prep::strip<MUON>(mats, nmats, tiles, blockIdx.x, partials, scale, eps, outputs, nscale, status, ticket,
                      nullptr, threadIdx.x, tile, red, &s_last, [] { __syncthreads(); });
}

// Long-side split: the summed FP32 Gram (s x s, leading dimension lda) into
// the padded BF16 operand A (sp x sp, zero outside s x s).
__global__ void __launch_bounds__(256) split_load_a_kernel(const float* __restrict__ A, int64_t lda, int s, int sp,
                                                           bf16* __restrict__ ah) {
    const int64_t n = (int64_t)sp * sp;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / sp), j = (int)(k % sp);
        ah[k] = __float2bfloat16_rn((i < s && j < s) ? A[(int64_t)i * lda + j] : 0.f);
    }
}

// Long-side split, BF16 path: the parts of tr(A) from which the square and
// update tiles compute d (the fused kernel's tr_a_sum / d_of), here from the
// summed FP32 Gram: one part per 32-row diagonal chunk, a butterfly over the
// chunk's 32 diagonal elements (rows >= s give 0), as the Gram epilogue forms
// them.
__global__ void __launch_bounds__(256) split_d_kernel(const float* __restrict__ A, int64_t lda, int s, int sp,
                                                      float* __restrict__ parts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < sp / 32; k += blockDim.x / 32) {
        const int i = 32 * k + lane;
        float d = (i < s) ? A[(int64_t)i * lda + i] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) parts[k] = d;
    }
}

}  // namespace

cudaError_t launch_split_d(const float* A, int64_t lda, int s, int sp, float* parts, cudaStream_t st) {
    split_d_kernel<<<1, 256, 0, st>>>(A, lda, s, sp, parts);
    return cudaGetLastError();
}

cudaError_t launch_split_load_a(const float* A, int64_t lda, int s, int sp, bf16* ah, cudaStream_t st) {
    const int64_t n = (int64_t)sp * sp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    split_load_a_kernel<<<blocks, 256, 0, st>>>(A, lda, s, sp, ah);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const DevMat* mats, int nmats, const TileTask* tiles, int ntiles, double* partials,
                           float scale, float eps, int outputs, float* nscale, int* status, int* counters,
                           int ncounters, unsigned* ticket, cudaStream_t st) {
    if (outputs & kPrepMuon)
        prepare_kernel<true><<<ntiles, 256, 0, st>>>(mats, nmats, tiles, partials, scale, eps, outputs, nscale,
                                                     status, counters, ncounters, ticket);
    else
        prepare_kernel<false><<<ntiles, 256, 0, st>>>(mats, nmats, tiles, partials, scale, eps, outputs, nscale,
                                                      status, counters, ncounters, ticket);
    return cudaGetLastError();
}

}  // namespace pe
