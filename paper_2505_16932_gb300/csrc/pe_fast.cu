// Fast polynomial iteration for rectangular matrices (Alg. 4, the appendix
// on rectangular matrices), FP32 path: the s x s products of a block.
//
// On the short side (X is s x L), a block of k polynomial steps takes
// Y = X X^T (+ shift I in the first block), Q_0 = I, and per step
// R_t = Q_{t-1}^T Y Q_{t-1}, Q_t = Q_{t-1} h_t(R_t) with
// h_t(r) = a_t + b_t r + c_t r^2; then X <- Q_k X. Y comes from the SIMT Gram
// kernel and X <- Q_k X from the SIMT update kernel (a = 0, B = Q_k); this
// file holds the s x s products in between:
//   fast_gemm_kernel<TA>  C = alpha op(A) B + beta E + gamma I (op(A) = A or
//                         A^T), one 128 x 128 output tile per block, every
//                         matrix of the call in one grouped launch; symmetric
//                         outputs (R, H, Q_1) on their upper tiles with
//                         mirrored stores; products with few tiles split
//                         along K into raw partial tiles, which
//   fast_reduce_kernel    sums in chunk order before the same epilogue;
//   fast_shift_kernel     Y += shift I on the first s diagonal entries.
// FP32 FMA accumulation (no TF32), 8 x 8 outputs per thread, double-buffered
// shared memory with rows padded by four floats, two blocks per SM; every
// operand is zero-padded to whole tiles.
#include <cuda_runtime.h>

#include "pe_internal.h"

namespace pe {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, PAD = 4;

// A: rows of op(A) K-contiguous (TA = false: a[i * lda + k]) or K rows of
// op(A)'s columns (TA = true: a[k * lda + i]); B: K rows (b[k * ldb + j])
template <bool TA>
__device__ __forceinline__ void load_ab(const GemmTask& t, int r0, int c0, int k0, int tid, float4 (&ra)[2],
                                        float4 (&rb)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = tid + h * 256;
        if (TA) {
            const int k = f >> 5, iq = (f & 31) * 4;
            ra[h] = *reinterpret_cast<const float4*>(t.a + (int64_t)(k0 + k) * t.lda + r0 + iq);
        } else {
            const int r = f >> 2, kq = (f & 3) * 4;
            ra[h] = *reinterpret_cast<const float4*>(t.a + (int64_t)(r0 + r) * t.lda + k0 + kq);
        }
        const int k = f >> 5, nq = (f & 31) * 4;
        rb[h] = *reinterpret_cast<const float4*>(t.b + (int64_t)(k0 + k) * t.ldb + c0 + nq);
    }
}

template <bool TA>
__device__ __forceinline__ void store_ab(float (*As)[BM + PAD], float (*Bs)[BN + PAD], int tid, const float4 (&ra)[2],
                                         const float4 (&rb)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = tid + h * 256;
        if (TA) {
            const int k = f >> 5, iq = (f & 31) * 4;
            *reinterpret_cast<float4*>(&As[k][iq]) = ra[h];
        } else {
            const int r = f >> 2, kq = (f & 3) * 4;
            As[kq + 0][r] = ra[h].x;
            As[kq + 1][r] = ra[h].y;
            As[kq + 2][r] = ra[h].z;
            As[kq + 3][r] = ra[h].w;
        }
        const int k = f >> 5, nq = (f & 31) * 4;
        *reinterpret_cast<float4*>(&Bs[k][nq]) = rb[h];
    }
}

template <bool TA>
__global__ void __launch_bounds__(256, 2) fast_gemm_kernel(const GemmTask* __restrict__ tasks, float alpha,
                                                           float beta, float gamma) {
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    const GemmTask t = tasks[blockIdx.x];
    const int r0 = t.tm * BM, c0 = t.tn * BN;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    float4 ra[2], rb[2];
    load_ab<TA>(t, r0, c0, t.k0, tid, ra, rb);
    store_ab<TA>(As[0], Bs[0], tid, ra, rb);
    __syncthreads();
    const int nk = t.kn / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load_ab<TA>(t, r0, c0, t.k0 + (kt + 1) * BK, tid, ra, rb);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float av[8], bv[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
            bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nk) store_ab<TA>(As[cur ^ 1], Bs[cur ^ 1], tid, ra, rb);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
            const int c = c0 + jh * 64 + tx * 4;
            float v[4];
            if (t.flags & kGemmPartial) {
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = acc[i][jh * 4 + j];
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = alpha * acc[i][jh * 4 + j];
                if (t.e) {
                    const float4 e4 = *reinterpret_cast<const float4*>(t.e + (int64_t)r * t.lde + c);
                    v[0] = fmaf(beta, e4.x, v[0]);
                    v[1] = fmaf(beta, e4.y, v[1]);
                    v[2] = fmaf(beta, e4.z, v[2]);
                    v[3] = fmaf(beta, e4.w, v[3]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (r == c + j) v[j] += gamma;
            }
            *reinterpret_cast<float4*>(t.c + (int64_t)r * t.ldc + c) = make_float4(v[0], v[1], v[2], v[3]);
            if ((t.flags & kGemmMirror) && !(t.flags & kGemmPartial) && t.tm != t.tn) {
#pragma unroll
                for (int j = 0; j < 4; ++j) t.c[(int64_t)(c + j) * t.ldc + r] = v[j];
            }
        }
    }
}

__global__ void __launch_bounds__(256) fast_reduce_kernel(const FastReduce* __restrict__ tasks, float alpha,
                                                          float beta, float gamma) {
    const FastReduce t = tasks[blockIdx.x];
    for (int q = threadIdx.x; q < BM * (BN / 4); q += 256) {
        const int r = t.tm * BM + (q >> 5), c = t.tn * BN + (q & 31) * 4;
        const float* p = t.part + (int64_t)r * t.ld + c;
        float4 acc = *reinterpret_cast<const float4*>(p);
        for (int k = 1; k < t.nsplit; ++k) {
            const float4 x = *reinterpret_cast<const float4*>(p + k * t.stride);
            acc.x += x.x;
            acc.y += x.y;
            acc.z += x.z;
            acc.w += x.w;
        }
        float v[4] = {alpha * acc.x, alpha * acc.y, alpha * acc.z, alpha * acc.w};
        if (t.e) {
            const float4 e4 = *reinterpret_cast<const float4*>(t.e + (int64_t)r * t.ld + c);
            v[0] = fmaf(beta, e4.x, v[0]);
            v[1] = fmaf(beta, e4.y, v[1]);
            v[2] = fmaf(beta, e4.z, v[2]);
            v[3] = fmaf(beta, e4.w, v[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (r == c + j) v[j] += gamma;
        *reinterpret_cast<float4*>(t.c + (int64_t)r * t.ld + c) = make_float4(v[0], v[1], v[2], v[3]);
        if ((t.flags & kGemmMirror) && t.tm != t.tn) {
#pragma unroll
            for (int j = 0; j < 4; ++j) t.c[(int64_t)(c + j) * t.ld + r] = v[j];
        }
    }
}

// Y += shift I on the first M.s diagonal entries of M.af (one block per matrix)
__global__ void fast_shift_kernel(const DevMat* __restrict__ mats, float shift) {
    const DevMat& M = mats[blockIdx.x];
    for (int i = threadIdx.x; i < M.s; i += blockDim.x) M.af[(int64_t)i * M.sp + i] += shift;
}

}  // namespace

cudaError_t launch_fast_gemm(const GemmTask* tasks, int ntasks, bool ta, float alpha, float beta, float gamma,
                             cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    if (ta) fast_gemm_kernel<true><<<ntasks, 256, 0, st>>>(tasks, alpha, beta, gamma);
    else fast_gemm_kernel<false><<<ntasks, 256, 0, st>>>(tasks, alpha, beta, gamma);
    return cudaGetLastError();
}

cudaError_t launch_fast_reduce(const FastReduce* tasks, int ntasks, float alpha, float beta, float gamma,
                               cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    fast_reduce_kernel<<<ntasks, 256, 0, st>>>(tasks, alpha, beta, gamma);
    return cudaGetLastError();
}

cudaError_t launch_fast_shift(const DevMat* mats, int nmats, float shift, cudaStream_t st) {
    if (nmats <= 0) return cudaSuccess;
    fast_shift_kernel<<<nmats, 256, 0, st>>>(mats, shift);
    return cudaGetLastError();
}

}  // namespace pe
