// Internal declarations shared by the host API and the kernels.
#pragma once

#include <stdint.h>

#include "../../include/polar_express.h"

namespace pe {

constexpr int kMaxSteps = 64;
constexpr int kMaxMatrices = 4096;
// Canonical padded layout: X is s x L (s = min(m,n)) padded to multiples of
// kPadS rows and kPadL columns with zeros; every GEMM then sees whole tiles.
constexpr int kPadS = 128;
constexpr int kPadL = 128;
// The prepare kernel takes one kPrepRows x kPrepCols strip of the padded
// layout per block (the last strip of a row may be kPadL wide); `ticket` and
// `nscale` hold one entry per descriptor and 64-row block of a pack (block k
// at index k nmats + descriptor), tickets zero between launches.
constexpr int kPrepRows = 64;
constexpr int kPrepCols = 256;
// BF16 matrices with a short side <= 64 are packed, up to kMaxPack of one
// shape, into one descriptor of kMaxPack 64-row blocks (block-diagonal A)
constexpr int kMaxPack = 4;

// sets the thread-local message returned by pe_last_error()
void set_last_error(const char* msg);

// host FP64 coefficient solver (pe_coeffs.cpp)
int coeffs_table(int degree, double l, int T, double safety, double cushion, unsigned flags,
                 double* coeffs, double* bounds, int* remez_iters, const char** why);

}  // namespace pe

#ifdef __CUDACC__
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace pe {

typedef __nv_bfloat16 bf16;

// Per-matrix device descriptor. All workspace pointers are canonical s x L
// (X) or s x s (A, B) padded row-major buffers with leading dimension Lp/sp.
struct DevMat {
    void* user;          // caller's m x n buffer (in/out)
    void* pack[kMaxPack - 1];  // pack: caller matrices 1 .. npack-1 of the same shape as `user`
                         // (s <= 64), whose canonical rows are 64 k .. 64 k + 63 of this
                         // descriptor's buffers (matrix 0 = `user` at rows 0 .. 63)
    int32_t npack;       // matrices in the descriptor (0: a plain descriptor)
    int64_t ld;          // caller's leading dimension (elements)
    int32_t m, n;        // caller's shape
    int32_t trans;       // 1 when m > n: X = G^T
    int32_t io;          // pe_io_type of the caller's buffer
    int32_t s, L;        // logical short / long side
    int32_t sp, Lp;      // padded sizes (multiples of kPadS / kPadL)
    int32_t part0, npart;  // prepare strips (norm partials) part0 .. part0 + npart; in a pack,
                           // block k's strips follow at part0 + k npart
    int32_t out_tma;       // 1 when the caller's buffer admits TMA stores
    float* xf;           // FP32 X (master; updated in place on the BF16x3 path)
    float* xf2;          // FP32 ping-pong partner (FP32 path)
    bf16* xh[2];         // BF16 X (hi part), ping-pong
    bf16* xl[2];         // BF16 X lo part (BF16x3), ping-pong
    int8_t* xq;          // BF16 path: byte of the next 8 mantissa bits of X
                         // below xh[cur] (see x_split), updated in place
    float* btr;          // BF16 path: tr(A) of the step in sp / 32 parts, one per 32-row
                         // diagonal chunk (written by the Gram epilogue), from which the
                         // square and update tiles compute d of the update
    int32_t ksplit;      // FP32 path: the Gram's reduction (length Lp) runs as ksplit chunks of
    int32_t kchunk;      // kchunk columns into the partial Grams gpart, summed in chunk order
                         // by the reduce kernel (ksplit <= 1: one pass straight into af)
    float* gpart;        // ksplit partial Grams, each sp x sp (tiles on and above the diagonal)
    float* af;           // FP32 A = X X^T (FP32, BF16x3)
    bf16* ah;            // BF16 A (hi)
    bf16* al;            // BF16 A lo (BF16x3)
    float* bfp;          // FP32 B (FP32 path)
    bf16* bh;            // BF16 B = bA + cA^2 (hi)
    bf16* bl;            // BF16 B lo (BF16x3)
    // fused Muon step (pe_muon_batched): `user` is the gradient G, `mom` the
    // momentum M <- beta M + (1 - beta) G (the iteration's input) and `w` the
    // weights W <- W - lr polar(M); all FP32 with the caller's shape and ld.
    float* mom;
    float* w;
    float beta, lr;
};

struct TileTask { int32_t mat, tm, tn, kind; };  // kind: 0 Gram, 1 A^2, 2 update

enum TileKind { kGram = 0, kSquare = 1, kApply = 2 };

// Which canonical buffers the prepare kernel fills.
enum PrepOut { kPrepF32 = 1, kPrepBF16 = 2, kPrepBF16Lo = 4, kPrepCode = 8,
               kPrepNoMom = 16,     // fused Muon: compute the momentum but leave M unchanged (tuning runs)
               kPrepMuon = 32,      // fused Muon: the kernel instantiation with the momentum update
               kPrepSkipPad = 64 }; // skip strips of padding rows (their buffers were zeroed once)

// Final store of element (i, l) of the canonical result X_T: into the
// caller's matrix, or for a fused Muon step W(i, l) <- W(i, l) - lr X_T(i, l).
__device__ __forceinline__ void out_user(const DevMat& M, int i, int l, float v) {
    void* user = M.user;
    if (M.npack && i >= 64) {   // matrix i / 64 of a pack
        const int k = i >> 6;
        if (k >= M.npack) return;
        user = M.pack[k - 1];
        i -= 64 * k;
    }
    if (i >= M.s || l >= M.L) return;
    const int64_t idx = M.trans ? (int64_t)l * M.ld + i : (int64_t)i * M.ld + l;
    if (M.w) M.w[idx] = __fadd_rn(M.w[idx], __fmul_rn(-M.lr, v));   // the rounding of a TMA reduce-add
    else if (M.io == PE_IO_BF16) reinterpret_cast<bf16*>(user)[idx] = __float2bfloat16_rn(v);
    else reinterpret_cast<float*>(user)[idx] = v;
}

// Compact master of X on the BF16 path: X is kept as hi = BF16 (the MMA
// operand) and one byte u holding the next 8 mantissa bits, i.e. x rounded to
// a 16-bit mantissa, in 3 bytes instead of the 6 of an FP32 copy plus a BF16
// operand. On the FP32 bit pattern b of x:
//   t  = b + 0x8080,   hi = t >> 16,   u = (t >> 8) & 0xFF
//   x' = bits^-1((hi << 16) + (u << 8) - 0x8000),   |x' - x| <= 2^-16 |x|.
// (hi rounds up from 0x7F80 of b's low half, not 0x8000, so that the signed
// residual code u - 128 = (b - (hi << 16) + 0x80) >> 8 never leaves a byte;
// u is that code in offset binary.) Zero maps to zero, signs never flip, and
// everything is integer arithmetic on the bit pattern (exact, deterministic).

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// t of x (see above): hi is its upper half, u its byte 1
__device__ __forceinline__ uint32_t x_split(float x) { return __float_as_uint(x) + 0x8080u; }

// hi of two elements from their t, the first in the low half
__device__ __forceinline__ uint32_t hi_pair(uint32_t t0, uint32_t t1) { return prmt(t0, t1, 0x7632u); }

// u of four elements (byte 1 of each t), the first in the low byte
__device__ __forceinline__ uint32_t code_quad(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3) {
    return prmt(prmt(t0, t1, 0x0051u), prmt(t2, t3, 0x0051u), 0x5410u);
}

// x' from hi << 16 and byte k of a code word: prmt moves the byte to byte 1
// with zeros elsewhere, i.e. u << 8
__device__ __forceinline__ float x_join(uint32_t hi32, uint32_t cw, int k) {
    const uint32_t sel = (4u << 12) | (4u << 8) | ((uint32_t)k << 4) | 4u;
    return __uint_as_float(hi32 + prmt(cw, 0u, sel) - 0x8000u);
}

// One 128 x 128 output tile of C = alpha op(A) B + beta E + gamma I (Alg. 4's
// s x s products; E may be null): row-major operands with leading
// dimensions, the reduction over k0 .. k0 + kn - 1 (multiples of 16).
// flags: kGemmMirror also stores the tile transposed (a symmetric output
// computed on its upper tiles, tm < tn); kGemmPartial stores the raw sum at
// c (a chunk of a split reduction; a FastReduce task applies the epilogue).
enum { kGemmMirror = 1, kGemmPartial = 2 };
struct GemmTask {
    const float* a;
    const float* b;
    const float* e;
    float* c;
    int32_t lda, ldb, lde, ldc;
    int32_t k0, kn, tm, tn;
    int32_t flags, pad0;
};

// One 128 x 128 output tile of a split reduction: C = alpha (sum of the
// nsplit partial tiles at part + k stride, in k order) + beta E + gamma I,
// mirrored when flags has kGemmMirror.
struct FastReduce {
    const float* part;
    const float* e;
    float* c;
    int64_t stride;
    int32_t nsplit, ld, tm, tn;
    int32_t flags, pad0;
};

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_prepare(const DevMat* mats, int nmats, const TileTask* tiles, int ntiles, double* partials,
                           float scale, float eps, int outputs, float* nscale, int* status, int* counters,
                           int ncounters, unsigned* ticket, cudaStream_t st);
cudaError_t launch_split_load_a(const float* A, int64_t lda, int s, int sp, bf16* ah, cudaStream_t st);
cudaError_t launch_split_d(const float* A, int64_t lda, int s, int sp, float* parts, cudaStream_t st);
cudaError_t launch_simt_phase(const DevMat* mats, const TileTask* tiles, int ntiles, int kind,
                              float a, float b, float c, int src, int last, int first,
                              const float* nscale, cudaStream_t st);
// Alg. 4 (FP32): the grouped s x s products (op(A) = A^T when ta) and the
// first block's shift Y += shift I
cudaError_t launch_fast_gemm(const GemmTask* tasks, int ntasks, bool ta, float alpha, float beta, float gamma,
                             cudaStream_t st);
cudaError_t launch_fast_reduce(const FastReduce* tasks, int ntasks, float alpha, float beta, float gamma,
                               cudaStream_t st);
cudaError_t launch_fast_shift(const DevMat* mats, int nmats, float shift, cudaStream_t st);
// FP32 path, matrices with ksplit > 1: A = s^2 (sum of the partial Grams in
// chunk order) on the tiles `tiles` (mat, tm, tn), mirrored below the diagonal
cudaError_t launch_simt_gram_reduce(const DevMat* mats, const TileTask* tiles, int ntiles, int first,
                                    const float* nscale, cudaStream_t st);

}  // namespace pe
#endif
