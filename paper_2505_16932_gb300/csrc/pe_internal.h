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
    int64_t ld;          // caller's leading dimension (elements)
    int32_t m, n;        // caller's shape
    int32_t trans;       // 1 when m > n: X = G^T
    int32_t io;          // pe_io_type of the caller's buffer
    int32_t s, L;        // logical short / long side
    int32_t sp, Lp;      // padded sizes (multiples of kPadS / kPadL)
    int32_t part0, npart;  // range of this matrix's prepare tiles (norm partials)
    int32_t out_tma;       // 1 when the caller's buffer admits TMA stores
    float* xf;           // FP32 X (master; updated in place on BF16 paths)
    float* xf2;          // FP32 ping-pong partner (FP32 path)
    bf16* xh[2];         // BF16 X (hi part), ping-pong
    bf16* xl[2];         // BF16 X lo part (BF16x3), ping-pong
    float* af;           // FP32 A = X X^T
    bf16* ah;            // BF16 A (hi)
    bf16* al;            // BF16 A lo (BF16x3)
    float* bfp;          // FP32 B (FP32 path)
    bf16* bh;            // BF16 B = bA + cA^2 (hi)
    bf16* bl;            // BF16 B lo (BF16x3)
};

struct TileTask { int32_t mat, tm, tn, kind; };  // kind: 0 Gram, 1 A^2, 2 update

enum TileKind { kGram = 0, kSquare = 1, kApply = 2 };

// Which canonical buffers the prepare kernel fills.
enum PrepOut { kPrepF32 = 1, kPrepBF16 = 2, kPrepBF16Lo = 4 };

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_prepare(const DevMat* mats, int nmats, const TileTask* tiles, int ntiles, double* partials,
                           float scale, float eps, int outputs, float* nscale, int* status, int* counters,
                           int ncounters, unsigned* ticket, cudaStream_t st);
cudaError_t launch_simt_phase(const DevMat* mats, const TileTask* tiles, int ntiles, int kind,
                              float a, float b, float c, int src, int last, int first,
                              const float* nscale, cudaStream_t st);

}  // namespace pe
#endif
