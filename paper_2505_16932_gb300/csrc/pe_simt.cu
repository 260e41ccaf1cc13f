// FP32 "plain method" path: SIMT FP32 FMA GEMMs (no TF32) for the three
// products of one polynomial step (Sec. 3.5 Horner form, App. A online code):
//   Gram    A = X X^T                     (upper-triangle tiles, mirrored)
//   square  B = b A + c A A               (upper-triangle tiles, mirrored)
//   update  X' = a X + B X                (ping-pong X buffers; the last step
//                                          writes the caller's layout)
// One grouped launch per product covers every matrix of the call: block
// i runs tile tiles[i] = (matrix, tile row, tile column). A Gram whose
// reduction is long (L > 4096) is cut into chunks along L (TileTask::kind
// carries the chunk index above its low byte): each block writes the
// chunk's partial product, and a reduce launch sums the partials in chunk
// order, so every output sums at most kchunk products in one accumulator
// (FP32 rounding error ~ sqrt(kchunk) u instead of ~ sqrt(L) u) and a
// tall-skinny Gram spreads over many blocks.
//
// 128 x 128 output tile per block, BK = 16, 256 threads, 8 x 8 outputs per
// thread as two 4 x 4 quadrants (rows ty*4 and 64 + ty*4, same for columns),
// double-buffered shared memory filled from registers prefetched one k-tile
// ahead; two blocks per SM (128 registers). Shared rows are padded by four
// floats, which keeps them 16-byte aligned for the vector reads and cuts the
// bank conflicts of the transposing stores from four-way to two-way. All operands are zero-padded to whole tiles, so there are no edge
// cases inside the product.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pe_internal.h"

namespace pe {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, PAD = 4;

struct Operands {
    const float* a;   // rows of the left operand, K contiguous
    int lda;
    const float* b;   // right operand: K-major rows (bk) or k x n rows (!bk)
    int ldb;
    int K;
};

template <bool kBKMajor>
__device__ __forceinline__ void load_tiles(const Operands& op, int r0, int c0, int k0, int tid,
                                           float4 (&ra)[2], float4 (&rb)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = tid + h * 256;
        const int r = f >> 2, kq = (f & 3) * 4;
        ra[h] = *reinterpret_cast<const float4*>(op.a + (int64_t)(r0 + r) * op.lda + k0 + kq);
        if (kBKMajor) {
            rb[h] = *reinterpret_cast<const float4*>(op.b + (int64_t)(c0 + r) * op.ldb + k0 + kq);
        } else {
            const int k = f >> 5, nq = (f & 31) * 4;
            rb[h] = *reinterpret_cast<const float4*>(op.b + (int64_t)(k0 + k) * op.ldb + c0 + nq);
        }
    }
}

template <bool kBKMajor>
__device__ __forceinline__ void store_tiles(float (*As)[BM + PAD], float (*Bs)[BN + PAD], int tid,
                                            const float4 (&ra)[2], const float4 (&rb)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = tid + h * 256;
        const int r = f >> 2, kq = (f & 3) * 4;
        As[kq + 0][r] = ra[h].x;
        As[kq + 1][r] = ra[h].y;
        As[kq + 2][r] = ra[h].z;
        As[kq + 3][r] = ra[h].w;
        if (kBKMajor) {
            Bs[kq + 0][r] = rb[h].x;
            Bs[kq + 1][r] = rb[h].y;
            Bs[kq + 2][r] = rb[h].z;
            Bs[kq + 3][r] = rb[h].w;
        } else {
            const int k = f >> 5, nq = (f & 31) * 4;
            *reinterpret_cast<float4*>(&Bs[k][nq]) = rb[h];
        }
    }
}

template <int kKind>
__global__ void __launch_bounds__(256, 2) simt_phase_kernel(const DevMat* __restrict__ mats,
                                                         const TileTask* __restrict__ tiles,
                                                         float ca, float cb, float cc, int src,
                                                         int last, int first, const float* __restrict__ nscale) {
    constexpr bool kBK = (kKind != kApply);
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    const TileTask tk = tiles[blockIdx.x];
    const DevMat& M = mats[tk.mat];
    const int r0 = tk.tm * BM, c0 = tk.tn * BN;
    const float* xs = src ? M.xf2 : M.xf;   // current X
    float* xd = src ? M.xf : M.xf2;         // next X
    Operands op;
    if (kKind == kGram) { op.a = xs; op.lda = M.Lp; op.b = xs; op.ldb = M.Lp; op.K = M.Lp; }
    else if (kKind == kSquare) { op.a = M.af; op.lda = M.sp; op.b = M.af; op.ldb = M.sp; op.K = M.sp; }
    else { op.a = M.bfp; op.lda = M.sp; op.b = xs; op.ldb = M.Lp; op.K = M.sp; }
    // split Gram: this block's chunk [kbeg, kend) of the reduction
    const bool part = (kKind == kGram) && M.ksplit > 1;
    const int kbeg = part ? (tk.kind >> 8) * M.kchunk : 0;
    const int kend = part ? min(op.K, kbeg + M.kchunk) : op.K;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra[2], rb[2];
    load_tiles<kBK>(op, r0, c0, kbeg, tid, ra, rb);
    store_tiles<kBK>(As[0], Bs[0], tid, ra, rb);
    __syncthreads();
    const int nk = (kend - kbeg) / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load_tiles<kBK>(op, r0, c0, kbeg + (kt + 1) * BK, tid, ra, rb);
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
        if (kt + 1 < nk) {
            store_tiles<kBK>(As[cur ^ 1], Bs[cur ^ 1], tid, ra, rb);
        }
        __syncthreads();
    }

    // epilogue; the first step applies the normalisation factor s
    // (A = s^2 X X^T, X_1 = s (a X + B X)) to the unscaled prepared X
    const float s0 = first ? nscale[tk.mat] : 1.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
            const int c = c0 + jh * 64 + tx * 4;
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = acc[i][jh * 4 + j];
            if (kKind == kGram && part) {
                // the chunk's partial product, unscaled (the reduce applies s^2)
                float* gp = M.gpart + (size_t)(tk.kind >> 8) * M.sp * M.sp;
                *reinterpret_cast<float4*>(gp + (int64_t)r * M.sp + c) = make_float4(v[0], v[1], v[2], v[3]);
            } else if (kKind == kGram) {
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] *= s0 * s0;
                *reinterpret_cast<float4*>(M.af + (int64_t)r * M.sp + c) = make_float4(v[0], v[1], v[2], v[3]);
                if (tk.tm != tk.tn) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) M.af[(int64_t)(c + j) * M.sp + r] = v[j];
                }
            } else if (kKind == kSquare) {
                const float4 a4 = *reinterpret_cast<const float4*>(M.af + (int64_t)r * M.sp + c);
                const float av4[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = fmaf(cb, av4[j], cc * v[j]);
                *reinterpret_cast<float4*>(M.bfp + (int64_t)r * M.sp + c) = make_float4(v[0], v[1], v[2], v[3]);
                if (tk.tm != tk.tn) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) M.bfp[(int64_t)(c + j) * M.sp + r] = v[j];
                }
            } else {
                const float4 x4 = *reinterpret_cast<const float4*>(xs + (int64_t)r * M.Lp + c);
                const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = s0 * fmaf(ca, xv[j], v[j]);
                if (last) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) out_user(M, r, c + j, v[j]);
                } else {
                    *reinterpret_cast<float4*>(xd + (int64_t)r * M.Lp + c) = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
        }
    }
}

// A = s^2 sum_k P_k over one 128 x 128 tile (mat, tm, tn) of a split Gram:
// partials summed in chunk order k = 0, 1, ..., the tile stored and, off the
// diagonal, mirrored
__global__ void __launch_bounds__(256) simt_gram_reduce_kernel(const DevMat* __restrict__ mats,
                                                               const TileTask* __restrict__ tiles, int first,
                                                               const float* __restrict__ nscale) {
    const TileTask tk = tiles[blockIdx.x];
    const DevMat& M = mats[tk.mat];
    const float s0 = first ? nscale[tk.mat] : 1.f;
    const size_t plane = (size_t)M.sp * M.sp;
    for (int e = threadIdx.x; e < BM * (BN / 4); e += 256) {
        const int r = tk.tm * BM + (e >> 5), c = tk.tn * BN + (e & 31) * 4;
        const float* p = M.gpart + (int64_t)r * M.sp + c;
        float4 acc = *reinterpret_cast<const float4*>(p);
        for (int k = 1; k < M.ksplit; ++k) {
            const float4 q = *reinterpret_cast<const float4*>(p + k * plane);
            acc.x += q.x;
            acc.y += q.y;
            acc.z += q.z;
            acc.w += q.w;
        }
        float v[4] = {acc.x * (s0 * s0), acc.y * (s0 * s0), acc.z * (s0 * s0), acc.w * (s0 * s0)};
        *reinterpret_cast<float4*>(M.af + (int64_t)r * M.sp + c) = make_float4(v[0], v[1], v[2], v[3]);
        if (tk.tm != tk.tn) {
#pragma unroll
            for (int j = 0; j < 4; ++j) M.af[(int64_t)(c + j) * M.sp + r] = v[j];
        }
    }
}

}  // namespace

cudaError_t launch_simt_gram_reduce(const DevMat* mats, const TileTask* tiles, int ntiles, int first,
                                    const float* nscale, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    simt_gram_reduce_kernel<<<ntiles, 256, 0, st>>>(mats, tiles, first, nscale);
    return cudaGetLastError();
}

cudaError_t launch_simt_phase(const DevMat* mats, const TileTask* tiles, int ntiles, int kind,
                              float a, float b, float c, int src, int last, int first,
                              const float* nscale, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    switch (kind) {
        case kGram:
            simt_phase_kernel<kGram><<<ntiles, 256, 0, st>>>(mats, tiles, a, b, c, src, last, first, nscale);
            break;
        case kSquare:
            simt_phase_kernel<kSquare><<<ntiles, 256, 0, st>>>(mats, tiles, a, b, c, src, last, first, nscale);
            break;
        default:
            simt_phase_kernel<kApply><<<ntiles, 256, 0, st>>>(mats, tiles, a, b, c, src, last, first, nscale);
            break;
    }
    return cudaGetLastError();
}

}  // namespace pe
