// Step S1 of the online stage (Alg. 1 online box; App. A online code):
//   nu = ||G||_F,  X_0 = G / (scale * nu + eps),
// written in the canonical short-side layout (X = G^T when m > n) and padded
// with zeros to whole tiles, in every precision the chosen path needs.
//
// Two grouped launches cover all matrices of a call:
//   pe_norm_partials  one block per row chunk, FP32 per thread, FP64 block sum
//   pe_prepare        one block per 64 x 64 canonical tile; sums the matrix's
//                     partials in a fixed order (deterministic), scales, casts,
//                     transposes and zero-pads.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "pe_internal.h"

namespace pe {

namespace {

__device__ __forceinline__ float load_in(const void* base, int io, int64_t idx) {
    if (io == PE_IO_BF16) return __bfloat162float(reinterpret_cast<const bf16*>(base)[idx]);
    return reinterpret_cast<const float*>(base)[idx];
}

__global__ void __launch_bounds__(256) norm_partials_kernel(const DevMat* __restrict__ mats,
                                                            const NormTask* __restrict__ tasks,
                                                            double* __restrict__ partials) {
    const NormTask tk = tasks[blockIdx.x];
    const DevMat& M = mats[tk.mat];
    float acc = 0.f;
    for (int r = tk.row0; r < tk.row1; ++r) {
        const int64_t rb = (int64_t)r * M.ld;
        for (int c = threadIdx.x; c < M.n; c += blockDim.x) {
            const float v = load_in(M.user, M.io, rb + c);
            acc = fmaf(v, v, acc);
        }
    }
    double d = (double)acc;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    __shared__ double red[8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        partials[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) prepare_kernel(const DevMat* __restrict__ mats,
                                                      const TileTask* __restrict__ tiles,
                                                      const double* __restrict__ partials,
                                                      float scale, float eps, int outputs,
                                                      int* __restrict__ status,
                                                      int* __restrict__ counters, int ncounters) {
    __shared__ float tile[64][65];
    __shared__ float s_inv;
    const TileTask tk = tiles[blockIdx.x];
    const DevMat& M = mats[tk.mat];
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < ncounters; i += blockDim.x) counters[i] = 0;
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double s = 0.0;
        for (int i = lane; i < M.npart; i += 32) s += partials[M.part0 + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double nu = sqrt(s);
            const double den = (double)scale * nu + (double)eps;
            float inv = (float)(1.0 / den);
            if (!isfinite(nu) || !(den > 0.0)) {
                atomicOr(status, 2);
                inv = 0.f;
            }
            s_inv = inv;
        }
    }
    __syncthreads();
    const float inv = s_inv;
    const int i0 = tk.tm * 64, l0 = tk.tn * 64;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    if (!M.trans) {
        // X[i][l] = G[i][l]
        for (int r = ty; r < 64; r += 4) {
            const int i = i0 + r, l = l0 + tx;
            float v = 0.f;
            if (i < M.s && l < M.L) v = load_in(M.user, M.io, (int64_t)i * M.ld + l) * inv;
            tile[r][tx] = v;
        }
    } else {
        // X[i][l] = G[l][i]; read G rows l with i contiguous, transpose in smem
        for (int r = ty; r < 64; r += 4) {
            const int l = l0 + r, i = i0 + tx;
            float v = 0.f;
            if (i < M.s && l < M.L) v = load_in(M.user, M.io, (int64_t)l * M.ld + i) * inv;
            tile[tx][r] = v;
        }
    }
    __syncthreads();
    for (int r = ty; r < 64; r += 4) {
        const int i = i0 + r, l = l0 + tx;
        const float v = tile[r][tx];
        const int64_t o = (int64_t)i * M.Lp + l;
        if (outputs & kPrepF32) M.xf[o] = v;
        if (outputs & (kPrepBF16 | kPrepBF16Lo)) {
            const bf16 h = __float2bfloat16_rn(v);
            M.xh[0][o] = h;
            if (outputs & kPrepBF16Lo) M.xl[0][o] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

}  // namespace

cudaError_t launch_norm_partials(const DevMat* mats, const NormTask* tasks, int ntasks,
                                 double* partials, cudaStream_t st) {
    norm_partials_kernel<<<ntasks, 256, 0, st>>>(mats, tasks, partials);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const DevMat* mats, const TileTask* tiles, int ntiles, const double* partials,
                           float scale, float eps, int outputs, int* status, int* counters,
                           int ncounters, cudaStream_t st) {
    prepare_kernel<<<ntiles, 256, 0, st>>>(mats, tiles, partials, scale, eps, outputs, status,
                                           counters, ncounters);
    return cudaGetLastError();
}

}  // namespace pe
