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

namespace pe {

namespace {

__device__ __forceinline__ float load_in(const void* base, int io, int64_t idx) {
    if (io == PE_IO_BF16) return __bfloat162float(reinterpret_cast<const bf16*>(base)[idx]);
    return reinterpret_cast<const float*>(base)[idx];
}

// four consecutive inputs of row `row` from column `col` of the caller's
// matrix at `src` (zero outside the matrix)
__device__ __forceinline__ float4 load4(const DevMat& M, const void* src, bool vec, int rows, int cols, int row,
                                        int col) {
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row >= rows) return r;
    const int64_t base = (int64_t)row * M.ld + col;
    if (vec && col + 3 < cols) {
        if (M.io == PE_IO_BF16) {
            const uint2 u = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const bf16*>(src) + base));
            const __nv_bfloat162 p0 = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
            const __nv_bfloat162 p1 = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
            r = make_float4(__low2float(p0), __high2float(p0), __low2float(p1), __high2float(p1));
        } else {
            r = __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(src) + base));
        }
        return r;
    }
    if (col + 0 < cols) r.x = load_in(src, M.io, base + 0);
    if (col + 1 < cols) r.y = load_in(src, M.io, base + 1);
    if (col + 2 < cols) r.z = load_in(src, M.io, base + 2);
    if (col + 3 < cols) r.w = load_in(src, M.io, base + 3);
    return r;
}

// Fused Muon step: M <- beta M + (1 - beta) G at the four inputs just read
// (same indices in M), stored back unless `store` is off; returns the new M,
// the value the iteration runs on.
__device__ __forceinline__ float4 momentum4(const DevMat& M, bool vec, int rows, int cols, int row, int col, float4 g,
                                            bool store) {
    if (row >= rows) return g;
    const float omb = 1.f - M.beta;
    const int64_t base = (int64_t)row * M.ld + col;
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vec && col + 3 < cols) {
        m = __ldcs(reinterpret_cast<const float4*>(M.mom + base));
    } else {
        if (col + 0 < cols) m.x = M.mom[base + 0];
        if (col + 1 < cols) m.y = M.mom[base + 1];
        if (col + 2 < cols) m.z = M.mom[base + 2];
        if (col + 3 < cols) m.w = M.mom[base + 3];
    }
    const float4 r = make_float4(fmaf(M.beta, m.x, __fmul_rn(omb, g.x)), fmaf(M.beta, m.y, __fmul_rn(omb, g.y)),
                                 fmaf(M.beta, m.z, __fmul_rn(omb, g.z)), fmaf(M.beta, m.w, __fmul_rn(omb, g.w)));
    if (store) {
        if (vec && col + 3 < cols) {
            *reinterpret_cast<float4*>(M.mom + base) = r;
        } else {
            if (col + 0 < cols) M.mom[base + 0] = r.x;
            if (col + 1 < cols) M.mom[base + 1] = r.y;
            if (col + 2 < cols) M.mom[base + 2] = r.z;
            if (col + 3 < cols) M.mom[base + 3] = r.w;
        }
    }
    // padding stays zero
    return make_float4(col + 0 < cols ? r.x : 0.f, col + 1 < cols ? r.y : 0.f, col + 2 < cols ? r.z : 0.f,
                       col + 3 < cols ? r.w : 0.f);
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void put4(const DevMat& M, int outputs, int64_t o, float4 v) {
    if (outputs & kPrepF32) *reinterpret_cast<float4*>(M.xf + o) = v;
    if (outputs & kPrepCode) {
        // BF16 path: hi and code of the compact master (x_split)
        const uint32_t t0 = x_split(v.x), t1 = x_split(v.y), t2 = x_split(v.z), t3 = x_split(v.w);
        *reinterpret_cast<uint2*>(M.xh[0] + o) = make_uint2(hi_pair(t0, t1), hi_pair(t2, t3));
        *reinterpret_cast<uint32_t*>(M.xq + o) = code_quad(t0, t1, t2, t3);
    } else if (outputs & (kPrepBF16 | kPrepBF16Lo)) {
        uint2 h;
        h.x = pack2(v.x, v.y);
        h.y = pack2(v.z, v.w);
        *reinterpret_cast<uint2*>(M.xh[0] + o) = h;
        if (outputs & kPrepBF16Lo) {
            const __nv_bfloat162 h0 = *reinterpret_cast<const __nv_bfloat162*>(&h.x);
            const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162*>(&h.y);
            uint2 l;
            l.x = pack2(v.x - __low2float(h0), v.y - __high2float(h0));
            l.y = pack2(v.z - __low2float(h1), v.w - __high2float(h1));
            *reinterpret_cast<uint2*>(M.xl[0] + o) = l;
        }
    }
}

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
    const TileTask tk = tiles[blockIdx.x];
    const DevMat& M = mats[tk.mat];
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < ncounters; i += blockDim.x) counters[i] = 0;
    }
    // canonical rows i0 .. i0 + 63 of the descriptor; in a pack they are
    // rows r0s = i0 - 64 blk .. of the pack's matrix blk
    const int blk = M.npack ? tk.tm : 0;
    const void* src = (blk == 0) ? M.user : (blk < M.npack ? M.pack[blk - 1] : nullptr);
    const int i0 = tk.tm * kPrepRows, l0 = tk.tn * kPrepCols;
    const int r0s = i0 - 64 * blk;
    const int tid = threadIdx.x;
    const int esz = (M.io == PE_IO_BF16) ? 2 : 4;
    const bool vec = (reinterpret_cast<uintptr_t>(src) % (4 * esz) == 0) && (M.ld % 4 == 0) &&
                     (!MUON || reinterpret_cast<uintptr_t>(M.mom) % 16 == 0);
    const bool mom_store = !(outputs & kPrepNoMom);
    float ss = 0.f;
    // all sixteen loads of a thread are issued before any store (the
    // compiler cannot move loads of G across stores that may alias it)
    float4 ld[16];
    if (!src || ((outputs & kPrepSkipPad) && r0s >= M.s)) {
        // every row of the strip is padding (or an empty block of a pack): the
        // workspace holds zeros there from the plan's creation on, and no step
        // ever writes anything else
    } else if (!M.trans) {
        // X[i][l] = G[i][l]; G is s x L. 64 threads per row, 4 rows per pass.
        const int c = (tid & 63) * 4, r0 = tid >> 6;
        const bool on = l0 + c < M.Lp;   // the last strip of a row may be 128 wide
        // interior strip of an FP32 matrix: sixteen unconditional vector loads
        const bool interior = vec && M.io != PE_IO_BF16 && r0s + kPrepRows <= M.s && l0 + kPrepCols <= M.L;
        if (interior) {
            const float* g = reinterpret_cast<const float*>(src) + (int64_t)(r0s + r0) * M.ld + l0 + c;
#pragma unroll
            for (int p = 0; p < 16; ++p) ld[p] = __ldcs(reinterpret_cast<const float4*>(g + (int64_t)4 * p * M.ld));
        } else {
#pragma unroll
            for (int p = 0; p < 16; ++p)
                ld[p] = on ? load4(M, src, vec, M.s, M.L, r0s + r0 + 4 * p, l0 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (MUON && on) {
#pragma unroll
            for (int p = 0; p < 16; ++p) ld[p] = momentum4(M, vec, M.s, M.L, r0s + r0 + 4 * p, l0 + c, ld[p], mom_store);
        }
        if (on) {
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                const float4 v = ld[p];
                ss = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, ss))));
                put4(M, outputs, (int64_t)(i0 + r0 + 4 * p) * M.Lp + l0 + c, v);
            }
        }
    } else {
        // X[i][l] = G[l][i]; G is L x s: read G rows l with i contiguous (16
        // threads per 64-float row segment), transpose 64 x 64 sub-tiles in smem
        const int rr = tid >> 4, c4 = (tid & 15) * 4;
        const bool interior = vec && M.io != PE_IO_BF16 && l0 + kPrepCols <= M.L && r0s + kPrepRows <= M.s;
        if (interior) {
            const float* g = reinterpret_cast<const float*>(src) + (int64_t)(l0 + rr) * M.ld + r0s + c4;
#pragma unroll
            for (int p = 0; p < 16; ++p) ld[p] = __ldcs(reinterpret_cast<const float4*>(g + (int64_t)16 * p * M.ld));
        } else {
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                const int l = l0 + rr + 16 * p;   // sub-tile p / 4, row rr + 16 (p % 4)
                ld[p] = (l < M.Lp) ? load4(M, src, vec, M.L, M.s, l, r0s + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (MUON) {
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                const int l = l0 + rr + 16 * p;
                if (l < M.Lp) ld[p] = momentum4(M, vec, M.L, M.s, l, r0s + c4, ld[p], mom_store);
            }
        }
#pragma unroll
        for (int k = 0; k < kPrepCols / 64; ++k) {
            if (l0 + 64 * k >= M.Lp) break;   // uniform across the block
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rr + 16 * q;
                const float4 v = ld[4 * k + q];
                ss = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, ss))));
                tile[r][c4 + 0] = v.x;
                tile[r][c4 + 1] = v.y;
                tile[r][c4 + 2] = v.z;
                tile[r][c4 + 3] = v.w;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rr + 16 * q;   // canonical row i0 + r, columns l0 + 64 k + c4 .. + 3
                const float4 v = make_float4(tile[c4 + 0][r], tile[c4 + 1][r], tile[c4 + 2][r], tile[c4 + 3][r]);
                put4(M, outputs, (int64_t)(i0 + r) * M.Lp + l0 + 64 * k + c4, v);
            }
            __syncthreads();
        }
    }
    // strip sum of squares: FP32 per thread, FP64 across the block, fixed order
    double d = (double)ss;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((tid & 31) == 0) red[tid >> 5] = d;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        partials[blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(&ticket[blk * nmats + tk.mat], 1u);
        s_last = (t == (unsigned)M.npart - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // last strip of this matrix to finish: its normalisation factor (the
    // matrix's strip partials in a fixed order: 32 strided lane sums, then a
    // butterfly), and the ticket reset for the next launch
    __threadfence();
    if (tid < 32) {
        const int lane = tid, m = blk * nmats + tk.mat;
        const int p0 = M.part0 + blk * M.npart;
        double s = 0.0;
        for (int i = lane; i < M.npart; i += 32) s += *((volatile double*)&partials[p0 + i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double nu = sqrt(s);
            // separate rounded multiply and add (no contraction), so that the
            // host computes the same value from the same sum (pe_split_set_norm)
            const double den = __dadd_rn(__dmul_rn((double)scale, nu), (double)eps);
            float inv = (float)(1.0 / den);
            if (!isfinite(nu) || !(den > 0.0)) {
                atomicOr(status, 2);
                inv = 0.f;
            }
            nscale[m] = inv;
            ticket[m] = 0u;
        }
    }
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
