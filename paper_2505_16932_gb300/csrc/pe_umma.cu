// BF16 / split-BF16 tensor-core path of one polynomial step (Sec. 3.5 Horner
// form; App. A online code), all on 128 x 256 output tiles:
//   Gram    A  = X X^T          tiles touching the upper triangle, mirrored
//   square  B  = b A + c A A    tiles touching the upper triangle, mirrored
//   update  X' = a X + B X
// on sm_103a tcgen05 tensor cores: operands staged in shared memory by TMA
// (128-byte swizzle, mbarrier ring), accumulators in TMEM (two 256-column
// buffers), warp-specialised roles:
//   warp 0     TMA producer (one lane)
//   warp 1     TMEM allocator + MMA issuer (one lane)
//   warps 2-9  epilogue, two warpgroups (one per half of the tile's
//              columns); each warp owns 32 tile rows (its TMEM lane quarter)
//              and works in 32 x 32 chunks.
//   warp 10    BF16 path: d of each square and update tile's update form,
//              computed ahead of the epilogue and handed over in shared
//              memory.
// BF16 epilogue: every chunk goes TMEM -> registers -> FP32 arithmetic ->
// swizzled shared-memory staging -> TMA bulk tensor stores; the epilogue's
// own operand (X for the update, A for the square) is fetched ahead by TMA
// into the warp's staging buffer. X is kept as its BF16 operand copy plus an
// 8-bit residual code (x_code), which carries the a X term at ~2^-16
// relative precision; b A takes the BF16 A the square reads anyway.
// Split-BF16 epilogue: the same arithmetic on FP32 X and A with direct
// global stores.
//
// The kernel is persistent and grouped: each CTA walks its own list of tiles
// (all matrices of the call, phase-ordered Gram -> square -> update). In the
// fused mode one launch runs the whole step, and a square/update tile waits
// (bounded, on a per-matrix counter) until every Gram/square tile of its
// matrix has been stored.
//
// Symmetric outputs: only 32 x 32 chunks on or above the diagonal are
// stored. Strictly-upper chunks are stored and mirrored; a diagonal chunk is
// symmetrised from its upper half. The FP32 copy of A (split-BF16 only)
// keeps the upper and diagonal chunks (the square epilogue reads nothing
// else).
//
// Split BF16 (BF16x3): every operand is x = hi + lo with hi = bf16(x),
// lo = bf16(x - hi); each k-step issues hi*hi + hi*lo + lo*hi into the same
// FP32 TMEM accumulator.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <queue>
#include <string>
#include <vector>

#include "pe_internal.h"
#include "pe_umma.h"

namespace pe {
namespace {

// Block layout: warp 0 producer, warp 1 MMA, then EW epilogue warps (8, or 12
// in the 2-SM kernel variant with more epilogue warps), then the d warp.
constexpr int threads_of(int ew) { return 64 + 32 * ew + 32; }
constexpr int kDRing = 16;                   // d hand-off slots (full / empty barriers each)
constexpr int kBM = 128;        // UMMA M
constexpr int kBN = 256;        // tile width (UMMA N, <= 256)
// The k-block BK (64 or 32 BF16 elements: one 128- or 64-byte swizzle row)
// is a template parameter; a smaller k-block gives more, smaller pipeline
// stages in the same shared memory.
constexpr uint64_t kDefaultWaitNs = 1000000000ull;  // 1 s

enum MapIdx {
    // operand maps, 128-byte swizzle: K-major boxes 64 x 128, MN-major 64 x 64
    kMapXK0 = 0, kMapXK1, kMapXM0, kMapXM1, kMapA, kMapB,
    kLo = 6,   // lo operand maps follow at +6 (BF16x3)
    // epilogue maps, 32 x 32 boxes: FP32 with 128-byte swizzle, BF16 with 64-byte
    // (kMapEXF, kMapEAF: reserved; kMapEXQ: codes of X, 32 x 32 bytes with
    // 32-byte swizzle)
    kMapEXF = 12, kMapEXH0, kMapEXH1, kMapEAF, kMapEAH, kMapEBH, kMapEOut, kMapEXQ,
    kMapsPerMat
};

struct StepArgs {
    const DevMat* mats;
    const CUtensorMap* maps;
    const int* off;
    const TileTask* tiles;
    const int* need;
    int* counters;
    int* status;
    float a, b, c;
    int step, cur, last, dependent, withhold;
    int cubic;          // c = 0 in every step: the Gram epilogue writes B = b A, no square tiles
    int nmats;          // descriptors (block k of a pack has nscale[k nmats + mat])
    uint64_t wait_ns;
    long long* prof;    // optional per-CTA cycle counters (debug)
    const float* nscale;  // per-matrix normalisation factor, applied in step 0
};

// ------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase. Returns false when the wait limit
// passes or another role of the CTA has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit,
                                          volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (globaltimer() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared::cluster address of the same offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// 2-SM form: the box lands in this CTA's shared memory, the bytes complete on
// an mbarrier that may live in the peer CTA (shared::cluster address).
__device__ __forceinline__ void tma_load_2d_cg2(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                                int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

__device__ __forceinline__ uint32_t ld_shared_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

// element-wise add of the box into global memory (f32, round to nearest)
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13,
// leading-dimension byte offset >> 4 in 16-29, stride-dimension byte offset
// >> 4 in 32-45, descriptor version 1 in bits 46-47, swizzle mode in 61-63
// (2 = 128-byte swizzle, 4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)swz << 61);
}

// Instruction descriptor, kind::f16: D format F32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), A K-major (bit 15 = 0), B major in bit 16,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N, bool b_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn_major ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_bf16_cg2(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// 2-SM commit: one arrival on the mbarrier at the shared::cluster address
// `bar_cluster` (this CTA's or the peer's) once every MMA issued so far by this
// thread has completed
__device__ __forceinline__ void umma_commit_cg2(uint32_t bar_cluster) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_cluster)
                 : "memory");
}

// the same barrier in both CTAs of the pair: one plain commit per CTA
__device__ __forceinline__ void umma_commit_cg2_pair(uint64_t* bar) {
    const uint32_t own = smem_u32(bar);
    umma_commit_cg2(own);
    umma_commit_cg2(mapa_rank(own, 1));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// named barrier of the N epilogue threads
template <int N>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }

// Bounded wait for a readiness counter (fused mode). On expiry the status
// word records a timeout and the caller proceeds: the launch always ends,
// with invalid results that pe_sync_status reports.
__device__ void wait_counter(const int* cnt, int target, uint64_t limit, int* status) {
    if (ld_acquire(cnt) >= target) return;
    const uint64_t t0 = globaltimer();
    unsigned ns = 32;
    while (ld_acquire(cnt) < target) {
        if (*reinterpret_cast<volatile int*>(status) & 1) return;
        if (globaltimer() - t0 > limit) {
            atomicOr(status, 1);
            return;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
}

// The BF16 update on the compact master X, X_b its BF16 part (the MMA
// operand): X' = (a + d) X + (B - d I) X_b, in exact arithmetic the step
// a X + B X for every d. B - d I is what the square epilogue rounds to BF16,
// and the update's rounding term is -(B - d I)(X - X_b). With d = 0 that term
// does not vanish once the singular values converge and B -> (1 - a) I, and
// the directions it rotates stay rotated. So once the mean of sigma^2,
// m = tr(A) / s, exceeds kConvergedMeanSq, d = b m + c m^2 (the mean of B's
// eigenvalues b sigma^2 + c sigma^4, with sigma^4 taken as m^2); before that
// d = 0, because the small singular directions, whose later growth amplifies
// their errors, fare better with B's own rounding.
constexpr float kConvergedMeanSq = 0.8f;

// d of the BF16 square and update (see kConvergedMeanSq) for the 64-row block
// blk of a pack (blk = 0 otherwise), from the parts of tr(A) the Gram
// epilogue left per 32-row diagonal chunk: lane k sums parts k, k + 32, ...
// in index order, a butterfly adds the lanes (every lane gets the same
// bits). The d warp computes it for each square and update tile ahead of
// the epilogue. split_d_kernel (pe_prep.cu) leaves the same parts for the
// long-side split.
__device__ __forceinline__ float tr_a_sum(const DevMat& M, int blk, int lane) {
    const int nsl = M.npack ? 2 : M.sp / 32;
    const float* p = M.btr + blk * nsl;
    float ta = 0.f;
    for (int j = lane; j < nsl; j += 32) ta += __ldcg(p + j);
    return ta;
}

__device__ __forceinline__ float d_of(float ta, const StepArgs& A, const DevMat& M) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ta += __shfl_xor_sync(0xffffffffu, ta, o);
    const float m = ta / (float)M.s;
    return (m > kConvergedMeanSq) ? fmaf(A.c * m, m, A.b * m) : 0.f;
}

// ------------------------------------------------------------ tile geometry

// TileTask::kind carries the product in its low bits.
constexpr int kKindMask = 3;

struct Geo {
    int kind, mat, tm, tn, bn, nkb;
    int mapA, mapB;      // hi operand maps
    int ya;              // A-operand row coordinate
    int b0;              // B-operand row (K-major) or column (MN-major) origin
    int col0;            // first output column of the tile
};

template <int BK>
__device__ __forceinline__ Geo tile_geo(const TileTask& tk, const DevMat& M, int cur) {
    Geo g;
    g.kind = tk.kind & kKindMask;
    g.mat = tk.mat;
    g.tm = tk.tm;
    g.tn = tk.tn;
    g.ya = tk.tm * kBM;
    g.b0 = tk.tn * kBN;
    g.col0 = g.b0;
    if (g.kind == kGram) {
        g.bn = min(kBN, M.sp - g.b0);
        g.nkb = M.Lp / BK;
        g.mapA = g.mapB = cur ? kMapXK1 : kMapXK0;
    } else if (g.kind == kSquare) {
        g.bn = min(kBN, M.sp - g.b0);
        g.nkb = M.sp / BK;
        g.mapA = g.mapB = kMapA;
    } else {
        g.bn = min(kBN, M.Lp - g.b0);
        g.nkb = M.sp / BK;
        g.mapA = kMapB;
        g.mapB = cur ? kMapXM1 : kMapXM0;
    }
    return g;
}

// chunk classes of a symmetric output
enum { kChunkLower = 0, kChunkDiag = 1, kChunkUpper = 2 };

__device__ __forceinline__ int chunk_class(int gi0, int gj0) {
    if (gj0 + 32 <= gi0) return kChunkLower;
    if (gj0 == gi0) return kChunkDiag;
    return kChunkUpper;
}

// ------------------------------------------------------ epilogue helpers

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a in the low half
    return *reinterpret_cast<uint32_t*>(&h);
}


// Swizzled 32 x 32 staging boxes. FP32 rows are 128 bytes (128-byte swizzle:
// 16-byte chunk c of row r lives at chunk c ^ (r & 7)); BF16 rows are 64
// bytes (64-byte swizzle: chunk c ^ ((r >> 1) & 3)). These are the layouts
// the TMA engine reads and writes for the epilogue tensor maps.
__device__ __forceinline__ uint32_t f32_off(int r, int c) {
    return r * 128 + ((((c >> 2) ^ (r & 7)) & 7) << 4) + (c & 3) * 4;
}
__device__ __forceinline__ uint32_t bf16_off(int r, int c) {
    return r * 64 + ((((c >> 3) ^ (r >> 1)) & 3) << 4) + (c & 7) * 2;
}

__device__ __forceinline__ void stage_f32_row(uint8_t* buf, int r, const float (&v)[32]) {
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4)
        *reinterpret_cast<float4*>(buf + f32_off(r, 4 * c4)) =
            make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
}

// Codes of X: 32-byte rows with 32-byte swizzle (16-byte chunk c of row r
// lives at chunk c ^ ((r >> 2) & 1)).
__device__ __forceinline__ uint32_t q8_off(int r, int c) {
    return r * 32 + ((((c >> 4) ^ (r >> 2)) & 1) << 4) + (c & 15);
}

// BF16 row of a box (64-byte swizzle) as FP32
__device__ __forceinline__ void read_bf16_row(const uint8_t* buf, int r, float (&v)[32]) {
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
        const uint4 u = *reinterpret_cast<const uint4*>(buf + bf16_off(r, 8 * c8));
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            v[8 * c8 + 2 * m] = __uint_as_float(w[m] << 16);   // low half: first element
            v[8 * c8 + 2 * m + 1] = __uint_as_float(w[m] & 0xFFFF0000u);
        }
    }
}

// X of a row from its hi box (BF16) at buf and its code box at buf + 2048
__device__ __forceinline__ void read_x_row(const uint8_t* buf, int r, float (&v)[32]) {
    const uint4 c0 = *reinterpret_cast<const uint4*>(buf + 2048 + q8_off(r, 0));
    const uint4 c1 = *reinterpret_cast<const uint4*>(buf + 2048 + q8_off(r, 16));
    const uint32_t cw[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
        const uint4 u = *reinterpret_cast<const uint4*>(buf + bf16_off(r, 8 * c8));
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 8 * c8 + 2 * m;
            v[j] = x_join(w[m] << 16, cw[j >> 2], j & 3);
            v[j + 1] = x_join(w[m] & 0xFFFF0000u, cw[(j + 1) >> 2], (j + 1) & 3);
        }
    }
}

// sum over the warp of each lane's element v[lane] (the diagonal of a
// diagonal chunk); every lane gets the same bits (xor butterfly)
__device__ __forceinline__ float warp_diag_sum(const float (&v)[32], int lane) {
    float d = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j)
        if (j == lane) d = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    return d;
}

// a row of X as hi (BF16 box at s_h) and code (box at s_q)
__device__ __forceinline__ void stage_x_row(uint8_t* s_h, uint8_t* s_q, int r, const float (&v)[32]) {
    uint32_t qw[8];
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
        uint32_t t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = x_split(v[8 * c8 + k]);
        *reinterpret_cast<uint4*>(s_h + bf16_off(r, 8 * c8)) =
            make_uint4(hi_pair(t[0], t[1]), hi_pair(t[2], t[3]), hi_pair(t[4], t[5]), hi_pair(t[6], t[7]));
        qw[2 * c8] = code_quad(t[0], t[1], t[2], t[3]);
        qw[2 * c8 + 1] = code_quad(t[4], t[5], t[6], t[7]);
    }
    *reinterpret_cast<uint4*>(s_q + q8_off(r, 0)) = make_uint4(qw[0], qw[1], qw[2], qw[3]);
    *reinterpret_cast<uint4*>(s_q + q8_off(r, 16)) = make_uint4(qw[4], qw[5], qw[6], qw[7]);
}

__device__ __forceinline__ void stage_bf16_row(uint8_t* buf, int r, const float (&v)[32]) {
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
        uint4 h;
        h.x = pack_bf16x2(v[8 * c8 + 0], v[8 * c8 + 1]);
        h.y = pack_bf16x2(v[8 * c8 + 2], v[8 * c8 + 3]);
        h.z = pack_bf16x2(v[8 * c8 + 4], v[8 * c8 + 5]);
        h.w = pack_bf16x2(v[8 * c8 + 6], v[8 * c8 + 7]);
        *reinterpret_cast<uint4*>(buf + bf16_off(r, 8 * c8)) = h;
    }
}

// transposed: element (c, r) of the box is v[c]
__device__ __forceinline__ void stage_f32_col(uint8_t* buf, int r, const float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 32; ++c) *reinterpret_cast<float*>(buf + f32_off(c, r)) = v[c];
}

__device__ __forceinline__ void stage_bf16_col(uint8_t* buf, int r, const float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 32; ++c) *reinterpret_cast<bf16*>(buf + bf16_off(c, r)) = __float2bfloat16_rn(v[c]);
}

// symmetric box from the upper half held by row r: (r, c) for c >= r and (c, r) for c > r
__device__ __forceinline__ void stage_bf16_sym(uint8_t* buf, int r, const float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const bf16 h = __float2bfloat16_rn(v[c]);
        if (c >= r) *reinterpret_cast<bf16*>(buf + bf16_off(r, c)) = h;
        if (c > r) *reinterpret_cast<bf16*>(buf + bf16_off(c, r)) = h;
    }
}

// ------------------------------------------ split-BF16 (register) epilogue

__device__ __forceinline__ void put_hl(bf16* hi, bf16* lo, int64_t idx, float v) {
    const bf16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ void store8_hl(bf16* hi, bf16* lo, const float* v) {
    uint4 h, l;
    float r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = v[q] - __bfloat162float(__float2bfloat16_rn(v[q]));
    h.x = pack_bf16x2(v[0], v[1]);
    h.y = pack_bf16x2(v[2], v[3]);
    h.z = pack_bf16x2(v[4], v[5]);
    h.w = pack_bf16x2(v[6], v[7]);
    l.x = pack_bf16x2(r[0], r[1]);
    l.y = pack_bf16x2(r[2], r[3]);
    l.z = pack_bf16x2(r[4], r[5]);
    l.w = pack_bf16x2(r[6], r[7]);
    *reinterpret_cast<uint4*>(hi) = h;
    *reinterpret_cast<uint4*>(lo) = l;
}

__device__ __forceinline__ void load32(float (&d)[32], const float* src) {
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(src + j);
        d[j] = x.x;
        d[j + 1] = x.y;
        d[j + 2] = x.z;
        d[j + 3] = x.w;
    }
}

// One 32-column chunk of row gi for the split-BF16 path; cls is the chunk's
// class for symmetric outputs.
__device__ __forceinline__ void chunk_hl(const Geo& g, const DevMat& M, const StepArgs& A, int gi, int col0,
                                         int cls, float s0, float (&v)[32], const float (&pre)[32]) {
    if (g.kind == kApply) {
        const int nxt = A.cur ^ 1;
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = s0 * fmaf(A.a, pre[j], v[j]);
        if (A.last) {
#pragma unroll
            for (int j = 0; j < 32; ++j) out_user(M, gi, col0 + j, v[j]);
            return;
        }
        float* xrow = M.xf + (int64_t)gi * M.Lp + col0;
#pragma unroll
        for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(xrow + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
#pragma unroll
        for (int j = 0; j < 32; j += 8)
            store8_hl(M.xh[nxt] + (int64_t)gi * M.Lp + col0 + j, M.xl[nxt] + (int64_t)gi * M.Lp + col0 + j, v + j);
        return;
    }
    if (g.kind == kSquare) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaf(A.b, pre[j], A.c * v[j]);
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= s0 * s0;
    }
    float* f32 = (g.kind == kGram) ? M.af : nullptr;
    bf16* hi = (g.kind == kGram) ? M.ah : M.bh;
    bf16* lo = (g.kind == kGram) ? M.al : M.bl;
    if (cls == kChunkUpper) {
        if (f32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4*>(f32 + (int64_t)gi * M.sp + col0 + j) =
                    make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
#pragma unroll
        for (int j = 0; j < 32; j += 8)
            store8_hl(hi + (int64_t)gi * M.sp + col0 + j, lo + (int64_t)gi * M.sp + col0 + j, v + j);
#pragma unroll
        for (int j = 0; j < 32; ++j) put_hl(hi, lo, (int64_t)(col0 + j) * M.sp + gi, v[j]);
    } else {   // diagonal chunk: symmetrise from the upper half
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int gj = col0 + j;
            if (gj >= gi) {
                const int64_t di = (int64_t)gi * M.sp + gj;
                if (f32) f32[di] = v[j];
                put_hl(hi, lo, di, v[j]);
            }
            if (gj > gi) {
                const int64_t mi = (int64_t)gj * M.sp + gi;
                if (f32) f32[mi] = v[j];
                put_hl(hi, lo, mi, v[j]);
            }
        }
    }
}

// -------------------------------------------------------------- kernel

// MODE 0: one CTA per 128 x 256 tile. MODE 2: 2-SM UMMA (cta_group::2) on
// 256 x 256 tiles, each CTA holding half of A (its 128 rows) and half of B
// (128 of the 256 columns). (MODE 1 is not used.)
template <int NS, int BK, int MODE = 0, int EW = 8>
struct Cfg {
    static constexpr int kEpiWarps = EW;
    static constexpr int kEpiThreads = 32 * EW;
    static constexpr int kDWarp = 2 + EW;   // computes d of the BF16 update ahead of the epilogue
    static constexpr int kThreads = threads_of(EW);
    static constexpr int kABytes = kBM * BK * 2;      // A tile of one k-block
    static constexpr int kBBytes = ((MODE == 2) ? kBN / 2 : kBN) * BK * 2;   // B tile (or half) of one k-block
    static constexpr int kAOps = (NS == 1) ? 1 : 2;   // stage: A hi | [A lo] | B hi | [B lo]
    static constexpr int kStage = kAOps * (kABytes + kBBytes);
    // (twelve epilogue warps take the shared memory of a fifth stage)
    static constexpr int kStages = (MODE == 2) ? (EW == 8 ? 5 : 4) : ((NS == 1) ? 3 : 2) * (64 / BK);
    // BF16 epilogue staging per warp: operand prefetch buffers of 3 KB (two,
    // fetched two chunks ahead; one in the 2-SM kernel, whose smem goes to a
    // fifth operand stage) and a 4 KB output box
    static constexpr int kNpf = (MODE == 2) ? 1 : 2;
    static constexpr int kWarpStage = 4096 + 3072 * kNpf;
    static constexpr uint32_t kSwzK = (BK == 64) ? 2u : 4u;   // K-major operand swizzle
    static constexpr uint32_t kSboK = 8 * BK * 2;             // 8 rows of one k-block
    static constexpr int kEpiOff = kStages * kStage;
    static constexpr int kBarOff = kEpiOff + ((NS == 1) ? EW * kWarpStage : 0);
    static_assert(kWarpStage % 1024 == 0, "staging boxes need 1024-byte alignment");
    static constexpr size_t kSmem = 1024 + kBarOff + 1024;   // barriers, TMEM slot, d ring
};

// Per-role cycle counters (debug profiling), slot k of CTA b at prof[32 b + k].
enum ProfSlot {
    kPTotal = 0, kPDepWait = 1, kPEmptyWait = 2, kPFullWait = 3, kPTEmptyWait = 4, kPTFullWait = 5,
    kPGramBusy = 6, kPSquareBusy = 7, kPApplyBusy = 8, kPEpiDepWait = 9, kPTiles = 10, kPProducer = 11,
    kPMma = 12,
    // update epilogue sub-steps: operand read + arithmetic, prefetch wait,
    // output staging, wait for the output box
    kPApRead = 13, kPApPf = 14, kPApMath = 15, kPApStore = 10, kPApFence = 16, kPApIssue = 17, kPApTmem = 18
};

// MODE = 2: clusters of two CTAs run one 256 x 256 tile with 2-SM UMMA; the
// even CTA issues the MMAs (M = 256), each CTA loads its half of A and B and
// reads its 128 accumulator rows from its own TMEM. NACC accumulators of 256
// columns are allocated (two give epilogue / MMA overlap).
// GF32: the long-side split's kernel, whose Gram writes the full FP32 A
// (DevMat::af); a separate instantiation keeps that path out of the others.
template <int NS, int BK, int MODE, int NACC, bool GF32 = false, int EW = 8>
__global__ void __launch_bounds__(threads_of(EW), 1) umma_step_kernel(const __grid_constant__ StepArgs A) {
    using C = Cfg<NS, BK, MODE, EW>;
    static_assert(C::kThreads == 64 + 32 * EW + 32, "block size of the configuration");
    static_assert(EW == 8 || (EW == 12 && NS == 1 && MODE == 2 && !GF32), "epilogue warps: 8, or 12 (2-SM BF16)");
    constexpr int kEpiWarps = C::kEpiWarps;
    constexpr int kEpiThreads = C::kEpiThreads;
    static_assert(MODE == 0 || MODE == 2, "kernel modes: 0 (1-SM tiles) and 2 (2-SM UMMA)");
    constexpr bool kCg2 = (MODE == 2);
    // the BF16 update's d (see kConvergedMeanSq): computed by the square and
    // update tiles from parts of tr(A) that the Gram tiles write, or, for the
    // long-side split (GF32), whose Grams are partial, split_d_kernel from the
    // summed Gram
    constexpr bool kUseD = (NS == 1);
    constexpr bool kPubD = (NS == 1) && !GF32;
    constexpr int kCols = 256 * NACC;
    constexpr int kABytes = C::kABytes;
    constexpr int kBBytes = C::kBBytes;
    constexpr int NST = C::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kBarOff);
    uint64_t* empty = full + NST;
    uint64_t* tfull = empty + NST;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint64_t* pfbar = drain + 1;            // two operand-prefetch barriers per epilogue warp
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pfbar + 2 * kEpiWarps);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint64_t* dfull = reinterpret_cast<uint64_t*>(tmem_slot + 2);   // d ring: slot written
    uint64_t* dempty = dfull + kDRing;                              // d ring: slot read by every epilogue warp
    float* dring = reinterpret_cast<float*>(dempty + kDRing);       // kDRing x 4 (a value per 64-row block)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t limit = A.wait_ns ? A.wait_ns : kDefaultWaitNs;
    const int crank = (MODE != 0) ? (int)cluster_rank() : 0;
    const int unit = (MODE != 0) ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int t_begin = A.off[unit];
    int t_end = A.off[unit + 1];
    // tile `it` of this CTA (2-SM: both CTAs of the pair read the same entry)
#define PE_TILE(it) (A.tiles[(it)])
    long long* prof = A.prof ? A.prof + 32 * blockIdx.x : nullptr;
    const long long k_t0 = clock64();

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], kCg2 ? 2 * kEpiWarps : kEpiThreads);
        }
        mbar_init(drain, 1);
        for (int w = 0; w < 2 * kEpiWarps; ++w) mbar_init(&pfbar[w], 1);
        for (int k = 0; k < kDRing; ++k) {
            mbar_init(&dfull[k], 1);
            mbar_init(&dempty[k], kEpiWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 1) {
        if (kCg2) {
            // one warp of each CTA of the pair performs the allocation collectively
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(kCols));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(kCols));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (MODE != 0) cluster_sync_all();   // both CTAs' barriers and TMEM exist before any cross-CTA traffic
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (kCg2) {
        // the MMA addresses both CTAs' TMEM at the even CTA's base: check they match
        const uint32_t peer = ld_shared_cluster_u32(mapa_rank(smem_u32(tmem_slot), (uint32_t)(crank ^ 1)));
        if (peer != tmem_base) {
            if (threadIdx.x == 0) atomicOr(A.status, 8);
            t_end = t_begin;   // do no work; both CTAs see the mismatch
        }
    }

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------ producer
        int stage = 0;
        uint32_t phase = 0;
        uint32_t issued = 0;   // bit s: stage s has been issued at least once
        uint32_t last_par = 0; // bit s: parity of the last issue of stage s
        bool ok = true;
        long long c_dep = 0, c_empty = 0;
        for (int it = t_begin; it < t_end && ok; ++it) {
            const TileTask tk = PE_TILE(it);
            const DevMat& M = A.mats[tk.mat];
            const Geo g = tile_geo<BK>(tk, M, A.cur);
            const CUtensorMap* mp = A.maps + (size_t)tk.mat * kMapsPerMat;
            if (A.dependent && g.kind != kGram) {
                const long long c0 = clock64();
                const int which = (g.kind == kSquare || A.cubic) ? 0 : 1;   // wait for A, or for B
                wait_counter(A.counters + 2 * g.mat + which, (A.step + 1) * A.need[2 * g.mat + which], limit,
                             A.status);
                fence_proxy_async_global();
                c_dep += clock64() - c0;
            }
            const uint32_t bbytes = (uint32_t)g.bn * BK * 2;
            // 2-SM: the even CTA's barrier receives both CTAs' halves of A and B
            const uint32_t tx = kCg2 ? (uint32_t)(2 * (kABytes + kBBytes)) : (uint32_t)C::kAOps * (kABytes + bbytes);
            const int ya2 = tk.tm * 2 * kBM + crank * kBM;     // 2-SM: this CTA's A rows
            const int bh2 = g.b0 + crank * (kBN / 2);          // 2-SM: this CTA's half of B
            for (int kb = 0; kb < g.nkb; ++kb) {
                const long long c0 = clock64();
                if (!mbar_wait(&empty[stage], phase ^ 1, limit, abort_flag)) { ok = false; break; }
                c_empty += clock64() - c0;
                const uint32_t sbase = smem_u32(smem + stage * C::kStage);
                const int kx = kb * BK;
                if (kCg2) {
                    if (crank == 0) mbar_expect_tx(&full[stage], tx);
                    const uint32_t fb = mapa_rank(smem_u32(&full[stage]), 0);
                    const uint32_t b_dst = sbase + kABytes;
                    tma_load_2d_cg2(sbase, mp + g.mapA, fb, kx, ya2);
                    if (g.kind == kApply) {
                        tma_load_2d_cg2(b_dst, mp + g.mapB, fb, bh2, kx);
                        tma_load_2d_cg2(b_dst + 64 * BK * 2, mp + g.mapB, fb, bh2 + 64, kx);
                    } else {
                        tma_load_2d_cg2(b_dst, mp + g.mapB, fb, kx, bh2);
                    }
                    issued |= 1u << stage;
                    last_par = (last_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == NST) { stage = 0; phase ^= 1; }
                    continue;
                }
                mbar_expect_tx(&full[stage], tx);
#pragma unroll
                for (int o = 0; o < C::kAOps; ++o) {
                    const int lo_off = o ? kLo : 0;
                    const uint32_t a_dst = sbase + o * kABytes;
                    const uint32_t b_dst = sbase + C::kAOps * kABytes + o * kBBytes;
                    tma_load_2d(a_dst, mp + g.mapA + lo_off, &full[stage], kx, g.ya);
                    if (g.kind == kApply) {
                        for (int j = 0; j < g.bn / 64; ++j)
                            tma_load_2d(b_dst + j * (64 * BK * 2), mp + g.mapB + lo_off, &full[stage],
                                        g.b0 + j * 64, kx);
                    } else {
                        for (int h = 0; h < g.bn / kBM; ++h)
                            tma_load_2d(b_dst + h * kABytes, mp + g.mapB + lo_off, &full[stage], kx,
                                        g.b0 + h * kBM);
                    }
                }
                issued |= 1u << stage;
                last_par = (last_par & ~(1u << stage)) | (phase << stage);
                if (++stage == NST) { stage = 0; phase ^= 1; }
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(A.status, 4);
            // let every issued copy land before the CTA can exit (2-SM: the
            // copies complete on the even CTA's barriers)
            if (!kCg2 || crank == 0)
                for (int s = 0; s < NST; ++s)
                    if (issued & (1u << s)) mbar_wait(&full[s], (last_par >> s) & 1u, limit, nullptr);
        }
        if (prof) {
            prof[kPDepWait] += c_dep;
            prof[kPEmptyWait] += c_empty;
            prof[kPProducer] += clock64() - k_t0;

        }
    } else if (warp == 1 && lane == 0 && (!kCg2 || crank == 0)) {
        // ------------------------------------------------------ MMA issuer
        int stage = 0;
        uint32_t phase = 0;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        long long c_full = 0, c_tempty = 0;
        for (int it = t_begin; it < t_end && ok; ++it) {
            const TileTask tk = PE_TILE(it);
            const DevMat& M = A.mats[tk.mat];
            const Geo g = tile_geo<BK>(tk, M, A.cur);
            long long c0 = clock64();
            if (!mbar_wait(&tempty[acc], acc_phase ^ 1, limit, abort_flag)) { ok = false; break; }
            c_tempty += clock64() - c0;
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + acc * 256;
            const bool mn = (g.kind == kApply);
            const uint32_t idesc = kCg2 ? idesc_bf16(2 * kBM, kBN, mn) : idesc_bf16(kBM, g.bn, mn);
            for (int kb = 0; kb < g.nkb; ++kb) {
                c0 = clock64();
                if (!mbar_wait(&full[stage], phase, limit, abort_flag)) { ok = false; break; }
                c_full += clock64() - c0;
                tc_fence_after();
                const uint32_t sbase = smem_u32(smem + stage * C::kStage);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
                    for (int p = 0; p < (NS == 1 ? 1 : 3); ++p) {
                        // products: hi*hi, hi*lo, lo*hi
                        const int ao = (p == 2) ? 1 : 0;
                        const int bo = (p == 1) ? 1 : 0;
                        const uint32_t a_addr = sbase + ao * kABytes + kk * 32;
                        const uint64_t adesc = sdesc(a_addr, 16, C::kSboK, C::kSwzK);
                        const uint32_t b_base = sbase + C::kAOps * kABytes + bo * kBBytes;
                        uint64_t bdesc;
                        if (mn) bdesc = sdesc(b_base + kk * 16 * 128, 64 * BK * 2, 1024, 2u);
                        else bdesc = sdesc(b_base + kk * 32, 16, C::kSboK, C::kSwzK);
                        if (kCg2) umma_bf16_cg2(d_tmem, adesc, bdesc, idesc, (kb | kk | p) != 0);
                        else umma_bf16(d_tmem, adesc, bdesc, idesc, (kb | kk | p) != 0);
                    }
                }
                if (kCg2) umma_commit_cg2_pair(&empty[stage]);
                else umma_commit(&empty[stage]);
                if (++stage == NST) { stage = 0; phase ^= 1; }
            }
            if (!ok) break;
            if (kCg2) umma_commit_cg2_pair(&tfull[acc]);
            else umma_commit(&tfull[acc]);
            if (++acc == NACC) { acc = 0; acc_phase ^= 1; }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(A.status, 4);
            if (kCg2) umma_commit_cg2(smem_u32(drain));
            else umma_commit(drain);
            mbar_wait(drain, 0, limit, nullptr);
        }
        if (prof) {
            prof[kPFullWait] += c_full;
            prof[kPTEmptyWait] += c_tempty;
            prof[kPMma] += clock64() - k_t0;
        }
    } else if (warp == C::kDWarp) {
        // ------------------------------------------------------ d of the BF16 update
        // Walks the CTA's tile list ahead of the epilogue: for each square and
        // update tile, once its matrix's Gram is complete (parts of tr(A)), d
        // per 64-row block of this CTA's rows into a ring slot; the epilogue
        // frees the slot after reading it.
        if (kUseD) {
            int slot = 0;
            uint32_t ph = 0;
            for (int it = t_begin; it < t_end; ++it) {
                const TileTask tk = PE_TILE(it);
                const DevMat& M = A.mats[tk.mat];
                if ((tk.kind & kKindMask) == kGram || !M.btr || A.cubic) continue;
                if (!mbar_wait(&dempty[slot], ph ^ 1, limit, abort_flag)) {
                    if (lane == 0) {
                        *abort_flag = 1;
                        atomicOr(A.status, 4);
                    }
                    break;
                }
                if (A.dependent) {   // the parts come from other CTAs' Gram tiles
                    const int* cnt = A.counters + 2 * tk.mat;
                    if (lane == 0) wait_counter(cnt, (A.step + 1) * A.need[2 * tk.mat], limit, A.status);
                    __syncwarp();
                    (void)ld_acquire(cnt);
                }
                const int row0 = kCg2 ? tk.tm * 2 * kBM + crank * kBM : tk.tm * kBM;
                for (int j = 0; j < (M.npack ? kBM / 64 : 1); ++j) {
                    const float dj = d_of(tr_a_sum(M, M.npack ? (row0 >> 6) + j : 0, lane), A, M);
                    if (lane == 0) dring[4 * slot + j] = dj;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&dfull[slot]);
                if (++slot == kDRing) {
                    slot = 0;
                    ph ^= 1;
                }
            }
        }
    } else if (warp >= 2) {
        // ------------------------------------------------------ epilogue
        const int ew = warp - 2;           // 0 .. EW - 1
        const int q = warp & 3;            // TMEM lane quarter = the warp's 32 tile rows
        const int grp = ew >> 2;           // column group of the tile (EW / 4 groups)
        constexpr int kGroups = EW / 4;
        // 32-column chunks per warp: 8 warps take a contiguous half of the
        // tile row each, 12 take every third chunk
        constexpr int kMaxCh = (kBN / 32 + kGroups - 1) / kGroups;
        const int etid = threadIdx.x - 64; // 0..255
        constexpr int NPF = C::kNpf;
        uint8_t* stg = smem + C::kEpiOff + ew * C::kWarpStage;
        // staging: two operand buffers (X hi at +0 and code at +2048, or
        // BF16 A) of 3 KB, then the output box: X hi + code (update), FP32
        // or BF16 result (last update), BF16 direct + mirror (symmetric)
        uint8_t* s_out = stg;                  // output box (4 KB, first: 1024-byte aligned)
        uint8_t* s_pf = stg + 4096;            // operand buffer b at s_pf + 3072 b
        // operand prefetches, issued and consumed in order: prefetch n uses
        // buffer n % NPF, whose barrier completes phase n / NPF
        uint32_t pf_issued = 0, pf_used = 0;
        int acc = 0;
        uint32_t acc_phase = 0;
        int dslot = 0;         // d ring slot of the next square / update tile
        uint32_t dph = 0;
        long long c_tfull = 0, c_dep = 0, c_gram = 0, c_sq = 0, c_ap = 0, c_rdx = 0, c_pf = 0, c_math = 0, c_st = 0, c_fn = 0,
                  c_is = 0, c_tm = 0;
        for (int it = t_begin; it < t_end; ++it) {
            const TileTask tk = PE_TILE(it);
            const DevMat& M = A.mats[tk.mat];
            const Geo g = tile_geo<BK>(tk, M, A.cur);
            const CUtensorMap* mp = A.maps + (size_t)tk.mat * kMapsPerMat;
            // the warp's first row (2-SM: this CTA holds rows 128 crank .. of the 256-row tile)
            const int gi0 = (kCg2 ? tk.tm * 2 * kBM + crank * kBM : g.tm * kBM) + q * 32;
            const int gi = gi0 + lane;
            // this warp's chunks: columns cb + i cs, i < nch
            const int nch = (kGroups == 2) ? g.bn / 64 : (g.bn / 32 - grp + kGroups - 1) / kGroups;
            const int cb = g.col0 + ((kGroups == 2) ? grp * nch * 32 : grp * 32);
            constexpr int cs = (kGroups == 2) ? 32 : 32 * kGroups;
            const bool sym = (g.kind != kApply);
            const bool needs_in = (g.kind != kGram);
            // step 0 runs on the unscaled prepared X and applies the
            // normalisation factor s: A = s^2 X X^T, X_1 = s (a X + B X)
            // (a warp's 32 rows lie in one 64-row block of a pack)
            const float s0 = (A.step == 0) ? A.nscale[(M.npack ? (gi0 >> 6) : 0) * A.nmats + g.mat] : 1.f;
            if (g.kind == kSquare && A.dependent) {   // A (FP32) comes from other CTAs
                const long long c0 = clock64();
                if (NS == 1) {
                    if (lane == 0) {
                        wait_counter(A.counters + 2 * g.mat, (A.step + 1) * A.need[2 * g.mat], limit, A.status);
                        fence_proxy_async_global();
                    }
                    __syncwarp();
                } else {
                    wait_counter(A.counters + 2 * g.mat, (A.step + 1) * A.need[2 * g.mat], limit, A.status);
                }
                c_dep += clock64() - c0;
            }
            // BF16 square and update: d comes from the d warp's ring (not for
            // c = 0 tables, whose B comes from the Gram)
            const bool use_d = kUseD && (g.kind != kGram) && M.btr && !A.cubic;
            // first chunk that this warp stores (symmetric outputs skip lower chunks)
            int first = 0;
            if (sym) {
                while (first < nch && chunk_class(gi0, cb + first * cs) == kChunkLower) ++first;
            }
            float pre[32];
            const float* in_g = (NS == 1) ? nullptr
                                : (g.kind == kApply) ? M.xf + (int64_t)gi * M.Lp : M.af + (int64_t)gi * M.sp;
            // BF16 path: the epilogue operand (update: X hi + code, square:
            // BF16 A) of each stored chunk is fetched by TMA NPF chunks ahead
            const CUtensorMap* in_map = mp + ((g.kind == kApply) ? (A.cur ? kMapEXH1 : kMapEXH0) : kMapEAH);
            const uint32_t in_bytes = (g.kind == kApply) ? 3072u : 2048u;
            auto prefetch = [&](int ch) {
                const int b = (NPF == 2) ? (int)(pf_issued & 1) : 0;
                if (lane == 0) {
                    const uint32_t dst = smem_u32(s_pf + b * 3072);
                    mbar_expect_tx(&pfbar[2 * ew + b], in_bytes);
                    tma_load_2d(dst, in_map, &pfbar[2 * ew + b], cb + ch * cs, gi0);
                    if (g.kind == kApply) tma_load_2d(dst + 2048, mp + kMapEXQ, &pfbar[2 * ew + b], cb + ch * cs, gi0);
                }
                ++pf_issued;
            };
            if (NS == 1) {
                if (needs_in) {
                    if (first < nch) prefetch(first);
                    if (NPF == 2 && first + 1 < nch) prefetch(first + 1);
                }
            } else if (needs_in && first < nch) {
                load32(pre, in_g + cb + first * cs);
            }
            long long c0 = clock64();
            if (!mbar_wait(&tfull[acc], acc_phase, limit, abort_flag)) {
                *abort_flag = 1;
                atomicOr(A.status, 4);
                break;
            }
            tc_fence_after();
            const long long c1 = clock64();
            c_tfull += c1 - c0;
            const uint32_t tbase = tmem_base + acc * 256 + ((uint32_t)(q * 32) << 16) + (cb - g.col0);
            float dtr = 0.f;
            if (use_d) {
                if (!mbar_wait(&dfull[dslot], dph, limit, abort_flag)) {
                    *abort_flag = 1;
                    atomicOr(A.status, 4);
                    break;
                }
                const int row0 = kCg2 ? tk.tm * 2 * kBM + crank * kBM : tk.tm * kBM;
                dtr = dring[4 * dslot + (M.npack ? (gi0 >> 6) - (row0 >> 6) : 0)];
                __syncwarp();
                if (lane == 0) mbar_arrive(&dempty[dslot]);
                if (++dslot == kDRing) {
                    dslot = 0;
                    dph ^= 1;
                }
            }
#pragma unroll
            for (int i = 0; i < kMaxCh; ++i) {
                if (i >= nch || i < first) continue;
                const int col0 = cb + i * cs;
                const int cls = sym ? chunk_class(gi0, col0) : kChunkUpper;
                if (cls == kChunkLower) continue;
                // pack: the Gram's blocks between different matrices stay zero
                // (never stored; the square then computes zeros there)
                if (g.kind == kGram && M.npack && (gi0 >> 6) != (col0 >> 6)) continue;
                // next stored chunk (for the prefetch)
                int nx = i + 1;
                if (sym)
                    while (nx < nch && chunk_class(gi0, cb + nx * cs) == kChunkLower) ++nx;
                float v[32];
                const bool sub = prof && g.kind == kApply;   // debug: update epilogue sub-steps
                long long s0c = sub ? clock64() : 0;
                tmem_ld32(tbase + i * cs, v);
                if (sub) { const long long t = clock64(); c_tm += t - s0c; s0c = t; }
                if (NS == 1) {
                    if (needs_in) {
                        const int b = (NPF == 2) ? (int)(pf_used & 1) : 0;
                        const uint32_t par = (NPF == 2) ? ((pf_used >> 1) & 1) : (pf_used & 1);
                        mbar_wait(&pfbar[2 * ew + b], par, limit, nullptr);
                        if (sub) { const long long t = clock64(); c_pf += t - s0c; s0c = t; }
                        if (g.kind == kApply) read_x_row(s_pf + b * 3072, lane, pre);
                        else read_bf16_row(s_pf + b * 3072, lane, pre);
                        ++pf_used;
                        if (NPF == 1) {
                            // single buffer: refill it for the next chunk as soon as
                            // every lane has read it (async-proxy write after
                            // generic-proxy reads: fence, then the issue)
                            fence_async_smem();
                            __syncwarp();
                            if (i + 1 < nch) prefetch(i + 1);
                        }
                    }
                    if (g.kind == kApply) {
                        // X' = (a + d) X + (B - d I) X_b (see kConvergedMeanSq)
                        const float ad = A.a + dtr;
                        if (A.step == 0) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) v[j] = s0 * fmaf(ad, pre[j], v[j]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j) v[j] = fmaf(ad, pre[j], v[j]);
                        }
                    } else if (g.kind == kSquare) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaf(A.b, pre[j], A.c * v[j]);
                        if (use_d && cls == kChunkDiag) {   // B - d I
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (j == lane) v[j] -= dtr;
                        }
                    } else {
                        // Gram: A = s^2 X X^T, or B = b s^2 X X^T when c = 0 throughout
                        const float gs = A.cubic ? A.b * s0 * s0 : s0 * s0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] *= gs;
                        if (kPubD && M.btr && !A.cubic && cls == kChunkDiag) {   // the parts of tr(A)
                            const float dg = warp_diag_sum(v, lane);
                            if (lane == 0) M.btr[gi0 >> 5] = dg;
                        }
                    }
                    if (sub) { const long long t = clock64(); c_rdx += t - s0c; s0c = t; }
                    if (GF32 && g.kind == kGram) {
                        // partial Gram of a long-side split: full symmetric FP32 A,
                        // row segment of this lane plus (coalesced) mirror columns
                        float* af = M.af;
                        if (cls == kChunkDiag) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int gj = col0 + j;
                                if (gj >= gi) af[(int64_t)gi * M.sp + gj] = v[j];
                                if (gj > gi) af[(int64_t)gj * M.sp + gi] = v[j];
                            }
                        } else {
                            float4* row = reinterpret_cast<float4*>(af + (int64_t)gi * M.sp + col0);
#pragma unroll
                            for (int j = 0; j < 8; ++j) row[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
#pragma unroll
                            for (int j = 0; j < 32; ++j) af[(int64_t)(col0 + j) * M.sp + gi] = v[j];
                        }
                        continue;
                    }
                    // the previous chunk's stores have read the output box
                    if (lane == 0) bulk_wait_read0();
                    __syncwarp();
                    if (sub) { const long long t = clock64(); c_st += t - s0c; s0c = t; }
                    const bool direct_out = !(g.kind == kApply && A.last && !M.out_tma);
                    if (g.kind == kApply && !A.last) {
                        stage_x_row(s_out, s_out + 2048, lane, v);
                    } else if (g.kind == kApply) {
                        if (M.out_tma) {
                            if (M.w) {   // fused Muon step: the box holds -lr X_T, reduce-added into W
#pragma unroll
                                for (int j = 0; j < 32; ++j) v[j] = __fmul_rn(-M.lr, v[j]);
                            }
                            if (M.io == PE_IO_BF16) {
                                if (M.trans) stage_bf16_col(s_out, lane, v); else stage_bf16_row(s_out, lane, v);
                            } else {
                                if (M.trans) stage_f32_col(s_out, lane, v); else stage_f32_row(s_out, lane, v);
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j) out_user(M, gi, col0 + j, v[j]);
                        }
                    } else if (cls == kChunkDiag) {
                        stage_bf16_sym(s_out, lane, v);
                    } else {
                        stage_bf16_row(s_out, lane, v);
                        stage_bf16_col(s_out + 2048, lane, v);
                    }
                    if (sub) { const long long t = clock64(); c_math += t - s0c; s0c = t; }
                    // one fence orders this chunk's generic reads of the operand
                    // buffer and writes of the output box before the async
                    // proxy's store of the box and refill of the buffer
                    fence_async_smem();
                    __syncwarp();
                    if (sub) { const long long t = clock64(); c_fn += t - s0c; s0c = t; }
                    if (lane == 0 && direct_out) {
                        if (g.kind == kApply && !A.last) {
                            tma_store_2d(mp + (A.cur ? kMapEXH0 : kMapEXH1), smem_u32(s_out), col0, gi0);
                            tma_store_2d(mp + kMapEXQ, smem_u32(s_out + 2048), col0, gi0);
                        } else if (g.kind == kApply) {
                            const int ox = M.trans ? gi0 : col0, oy = M.trans ? col0 : gi0;
                            if (M.w) tma_reduce_add_2d(mp + kMapEOut, smem_u32(s_out), ox, oy);
                            else tma_store_2d(mp + kMapEOut, smem_u32(s_out), ox, oy);
                        } else {
                            const CUtensorMap* hm = mp + ((g.kind == kGram && !A.cubic) ? kMapEAH : kMapEBH);
                            tma_store_2d(hm, smem_u32(s_out), col0, gi0);
                            if (cls != kChunkDiag) tma_store_2d(hm, smem_u32(s_out + 2048), gi0, col0);
                        }
                        bulk_commit();
                    }
                    if (NPF == 2 && needs_in && i + 2 < nch) prefetch(i + 2);
                    if (sub) { __syncwarp(); c_is += clock64() - s0c; }
                } else {
                    float nxt_pre[32];
                    if (needs_in && nx < nch) load32(nxt_pre, in_g + cb + nx * cs);
                    chunk_hl(g, M, A, gi, col0, cls, s0, v, pre);
                    if (needs_in && nx < nch) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) pre[j] = nxt_pre[j];
                    }
                }
            }
            tc_fence_before();
            if (kCg2) {
                // one arrival per warp on the even CTA's accumulator-empty barrier
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(mapa_rank(smem_u32(&tempty[acc]), 0));
            } else {
                mbar_arrive(&tempty[acc]);
            }
            if (A.dependent && sym) {
                if (NS == 1 && lane == 0) {
                    bulk_wait0();
                    fence_proxy_async_global();
                }
                __threadfence();
                epi_bar<kEpiThreads>();
                if (etid == 0 && !(g.kind == kGram && g.mat == A.withhold))
                    red_release_add(A.counters + 2 * g.mat + (g.kind == kSquare ? 1 : 0), 1);
            }
            const long long dc = clock64() - c1;
            if (g.kind == kGram) c_gram += dc;
            else if (g.kind == kSquare) c_sq += dc;
            else c_ap += dc;
            if (++acc == NACC) { acc = 0; acc_phase ^= 1; }
        }
        // operand prefetches still in flight (a tile left early) land before exit
        for (; pf_used < pf_issued; ++pf_used) {
            if (NPF == 2) mbar_wait(&pfbar[2 * ew + (pf_used & 1)], (pf_used >> 1) & 1, limit, nullptr);
            else mbar_wait(&pfbar[2 * ew], pf_used & 1, limit, nullptr);
        }
        if (NS == 1 && lane == 0) bulk_wait0();
        if (prof && etid == 0) {
            prof[kPTFullWait] += c_tfull;
            prof[kPEpiDepWait] += c_dep;
            prof[kPGramBusy] += c_gram;
            prof[kPSquareBusy] += c_sq;
            prof[kPApplyBusy] += c_ap;
            prof[kPApRead] += c_rdx;
            prof[kPApPf] += c_pf;
            prof[kPApMath] += c_math;
            prof[kPApStore] += c_st;
            prof[kPApFence] += c_fn;
            prof[kPApIssue] += c_is;
            prof[kPApTmem] += c_tm;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (MODE != 0) cluster_sync_all();   // the peer no longer touches this CTA
#undef PE_TILE
    if (prof && threadIdx.x == 0) prof[kPTotal] += clock64() - k_t0;
    if (warp == 1) {
        tc_fence_after();
        if (kCg2)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kCols));
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kCols));
    }
}

// ----------------------------------------------------------------- host

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn(std::string* err) {
    static EncodeTiledFn fn = nullptr;
    if (fn) return fn;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
        *err = "cuTensorMapEncodeTiled is not available from the driver";
        return nullptr;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
    return fn;
}

// 2-D row-major map: rows x cols, row pitch in bytes, box = box_cols x box_rows.
bool make_map(EncodeTiledFn enc, CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int64_t pitch,
              int box_rows, int box_cols, CUtensorMapDataType dt, CUtensorMapSwizzle sw) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, dt, 2,
                     const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct HostTile {
    TileTask t;
    double cost;
};

// Tiles of one matrix. Symmetric products keep the 128 x 256 tiles that
// reach the upper triangle (column end > row start).
void tiles_of(const DevMat& M, int i, std::vector<HostTile>* ph, bool cubic) {
    const int tm = M.sp / kBM;
    const int ts = (M.sp + kBN - 1) / kBN;
    for (int a = 0; a < tm; ++a)
        for (int b = 0; b < ts; ++b) {
            const int bn = std::min(kBN, M.sp - b * kBN);
            if (b * kBN + bn <= a * kBM) continue;
            ph[kGram].push_back(HostTile{TileTask{i, a, b, kGram}, (double)kBM * bn * M.Lp});
            if (!cubic) ph[kSquare].push_back(HostTile{TileTask{i, a, b, kSquare}, (double)kBM * bn * M.sp});
        }
    const int tl = (M.Lp + kBN - 1) / kBN;
    for (int a = 0; a < tm; ++a)
        for (int b = 0; b < tl; ++b) {
            const int bn = std::min(kBN, M.Lp - b * kBN);
            ph[kApply].push_back(HostTile{TileTask{i, a, b, kApply}, (double)kBM * bn * M.sp});
        }
}

// Tile order inside a phase. Mode 0: longest first. Mode 1: by matrix
// (largest first), then in column groups of 8 tile columns, row-major inside
// a group, so that the tiles running at one time share few operand blocks.
void sort_phase(std::vector<HostTile>& v, int mode, const std::vector<double>& mat_cost) {
    if (mode == 0) {
        std::stable_sort(v.begin(), v.end(), [](const HostTile& x, const HostTile& y) { return x.cost > y.cost; });
        return;
    }
    std::stable_sort(v.begin(), v.end(), [&](const HostTile& x, const HostTile& y) {
        if (x.t.mat != y.t.mat) {
            const double cx = mat_cost[x.t.mat], cy = mat_cost[y.t.mat];
            if (cx != cy) return cx > cy;
            return x.t.mat < y.t.mat;
        }
        if (x.t.tn / 8 != y.t.tn / 8) return x.t.tn / 8 < y.t.tn / 8;
        if (x.t.tm != y.t.tm) return x.t.tm < y.t.tm;
        return x.t.tn < y.t.tn;
    });
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// Orders of the fused list. 0, 1: phase-major (every Gram tile, then every
// square tile, then every update tile) with the in-phase order of
// sort_phase mode 0 / 1. 2, 3, 4: lagged interleave: a tile of phase k of the
// matrix of cost rank r gets the key r + D k (D = 4, 8, 16), so that update
// tiles (memory-heavy) of early matrices run beside Gram tiles
// (compute-heavy) of later ones. Every order lists a matrix's phases in
// dependency order, which is what the readiness waits need for progress.

namespace {

struct Unit {
    TileTask t;
    double cost;
};

std::vector<Unit> make_units(const std::vector<TileTask>& tiles, const std::vector<double>& cost) {
    std::vector<Unit> u;
    for (size_t i = 0; i < tiles.size(); ++i) u.push_back(Unit{tiles[i], cost[i]});
    return u;
}

void sort_units(std::vector<Unit>& v, int mode, const std::vector<double>& mat_cost) {
    std::vector<HostTile> h;
    for (size_t i = 0; i < v.size(); ++i) {
        TileTask key = v[i].t;
        key.kind = (int)i;   // carry the unit index through the sort
        h.push_back(HostTile{key, v[i].cost});
    }
    sort_phase(h, mode, mat_cost);
    std::vector<Unit> out;
    for (const HostTile& x : h) out.push_back(v[x.t.kind]);
    v.swap(out);
}

void lpt_units(const std::vector<Unit>& order, int groups, std::vector<int>* off, std::vector<TileTask>* out) {
    std::vector<std::vector<int>> per(groups);
    typedef std::pair<double, int> Load;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int c = 0; c < groups; ++c) pq.push(Load(0.0, c));
    for (size_t i = 0; i < order.size(); ++i) {
        Load l = pq.top();
        pq.pop();
        per[l.second].push_back((int)i);
        l.first += order[i].cost + 2.0e5;
        pq.push(l);
    }
    off->assign(groups + 1, 0);
    out->clear();
    int n = 0;
    for (int c = 0; c < groups; ++c) {
        (*off)[c] = n;
        for (int i : per[c]) {
            out->push_back(order[i].t);
            ++n;
        }
    }
    (*off)[groups] = n;
}

}  // namespace

int umma_schedule(UmmaPlan* P, int order, std::string* err) {
    const bool cg2 = P->mode >= 2;     // one 256 x 256 tile per unit
    const int inphase = (order == 1) ? 1 : 0;
    std::vector<Unit> ph[3];
    for (int k = 0; k < 3; ++k) {
        if (cg2) ph[k] = make_units(P->ph2_t[k], P->ph2_c[k]);
        else ph[k] = make_units(P->ph_t[k], P->ph_c[k]);
        sort_units(ph[k], inphase, P->mat_cost);
    }
    std::vector<Unit> fused;
    if (order <= 1) {
        for (int k = 0; k < 3; ++k) fused.insert(fused.end(), ph[k].begin(), ph[k].end());
    } else {
        const int lag = (order == 2) ? 4 : (order == 3) ? 8 : 16;
        const int count = (int)P->mat_cost.size();
        std::vector<int> idx(count), rank(count);
        for (int i = 0; i < count; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return P->mat_cost[a] > P->mat_cost[b]; });
        for (int r = 0; r < count; ++r) rank[idx[r]] = r;
        struct Keyed { long key; int phase; size_t pos; };
        std::vector<Keyed> all;
        for (int k = 0; k < 3; ++k)
            for (size_t i = 0; i < ph[k].size(); ++i)
                all.push_back(Keyed{(long)rank[ph[k][i].t.mat] + (long)lag * k, k, i});
        std::stable_sort(all.begin(), all.end(), [](const Keyed& a, const Keyed& b) {
            if (a.key != b.key) return a.key < b.key;
            if (a.phase != b.phase) return a.phase < b.phase;
            return a.pos < b.pos;
        });
        for (const Keyed& k : all) fused.push_back(ph[k.phase][k.pos]);
    }
    const int cap = (P->mode == 3) ? P->max_clusters3 : cg2 ? P->max_clusters2 : P->sms;   // scheduling groups
    P->ntiles = (int)fused.size();
    const int groups = std::max(1, std::min(cap, P->ntiles));
    P->grid = cg2 ? 2 * groups : groups;
    std::vector<int> off;
    std::vector<TileTask> list;
    lpt_units(fused, groups, &off, &list);
    cudaError_t e = cudaMemcpy(P->tiles, list.data(), sizeof(TileTask) * list.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->tile_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        std::vector<int> poff;
        std::vector<TileTask> plist;
        const int g = std::max(1, std::min(cap, (int)ph[k].size()));
        lpt_units(ph[k], g, &poff, &plist);
        P->grid_phase[k] = ph[k].empty() ? 0 : (cg2 ? 2 * g : g);
        if (!plist.empty())
            e = cudaMemcpy(P->ph_tiles[k], plist.data(), sizeof(TileTask) * plist.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P->ph_off[k], poff.data(), sizeof(int) * poff.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        *err = std::string("uploading the tile schedule: ") + cudaGetErrorString(e);
        return PE_ECUDA;
    }
    P->order = order;
    return PE_OK;
}

size_t umma_workspace_bytes(const DevMat* mats, int count) {
    size_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        const size_t tm = mats[i].sp / kBM;
        const size_t ts = (mats[i].sp + kBN - 1) / kBN;
        const size_t tl = (mats[i].Lp + kBN - 1) / kBN;
        tiles += 2 * tm * ts + tm * tl;
    }
    size_t b = 0;
    b += align_up(sizeof(CUtensorMap) * kMapsPerMat * count, 1024);
    b += 2 * align_up(sizeof(TileTask) * (tiles + 2), 256);   // fused + phased lists
    b += 4 * align_up(sizeof(int) * (4096 + 1), 256);         // CSR offsets (grid <= 4096)
    b += 2 * align_up(sizeof(int) * 2 * count, 256);
    return b + 4096;
}

int umma_build(UmmaPlan* P, DevMat* mats, DevMat* d_mats, int count, int dtype, int sms, char* ws,
               size_t ws_bytes, int* counters, bool tune, std::string* err) {
    (void)tune;
    EncodeTiledFn enc = encode_fn(err);
    if (!enc) return PE_EUNSUPPORTED;
    P->count = count;
    P->dtype = dtype;
    P->nsplit = (dtype == PE_BF16X3) ? 3 : 1;
    P->d_mats = d_mats;
    P->counters = counters;
    std::vector<CUtensorMap> maps(kMapsPerMat * count);
    memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    std::vector<HostTile> ph[3];
    std::vector<int> need(2 * count);
    const CUtensorMapSwizzle S128 = CU_TENSOR_MAP_SWIZZLE_128B, S64 = CU_TENSOR_MAP_SWIZZLE_64B;
    const CUtensorMapDataType BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              U8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    for (int i = 0; i < count; ++i) {
        DevMat& M = mats[i];
        CUtensorMap* mp = maps.data() + (size_t)i * kMapsPerMat;
        bool ok = true;
        const int64_t xp = (int64_t)M.Lp * 2, sp2 = (int64_t)M.sp * 2;
        const int bk = P->bk;
        const CUtensorMapSwizzle SK = (bk == 64) ? S128 : S64;   // K-major operand boxes: bk x 128
        for (int lo = 0; lo < (P->nsplit == 3 ? 2 : 1); ++lo) {
            bf16* const* x = lo ? M.xl : M.xh;
            const int o = lo ? kLo : 0;
            ok &= make_map(enc, mp + o + kMapXK0, x[0], M.sp, M.Lp, xp, kBM, bk, BF, SK);
            ok &= make_map(enc, mp + o + kMapXK1, x[1], M.sp, M.Lp, xp, kBM, bk, BF, SK);
            ok &= make_map(enc, mp + o + kMapXM0, x[0], M.sp, M.Lp, xp, bk, 64, BF, S128);
            ok &= make_map(enc, mp + o + kMapXM1, x[1], M.sp, M.Lp, xp, bk, 64, BF, S128);
            ok &= make_map(enc, mp + o + kMapA, lo ? M.al : M.ah, M.sp, M.sp, sp2, kBM, bk, BF, SK);
            ok &= make_map(enc, mp + o + kMapB, lo ? M.bl : M.bh, M.sp, M.sp, sp2, kBM, bk, BF, SK);
        }
        if (P->nsplit == 1) {
            ok &= make_map(enc, mp + kMapEXQ, M.xq, M.sp, M.Lp, (int64_t)M.Lp, 32, 32, U8,
                           CU_TENSOR_MAP_SWIZZLE_32B);
            ok &= make_map(enc, mp + kMapEXH0, M.xh[0], M.sp, M.Lp, xp, 32, 32, BF, S64);
            ok &= make_map(enc, mp + kMapEXH1, M.xh[1], M.sp, M.Lp, xp, 32, 32, BF, S64);
            ok &= make_map(enc, mp + kMapEAH, M.ah, M.sp, M.sp, sp2, 32, 32, BF, S64);
            ok &= make_map(enc, mp + kMapEBH, M.bh, M.sp, M.sp, sp2, 32, 32, BF, S64);
        }
        if (!ok) {
            *err = "cuTensorMapEncodeTiled failed for matrix " + std::to_string(i);
            return PE_ECUDA;
        }
        // the caller's buffer takes TMA stores when it is 16-byte aligned, its
        // pitch is a multiple of 16 bytes and so is its row (n elements): a
        // box that crosses the right edge of the tensor is written in whole
        // 16-byte granules, so a row ending inside a granule would get the
        // padding columns' zeros written past its end (into the caller's gap
        // between rows); such matrices take element-wise stores (out_user)
        const int esz = (M.io == PE_IO_BF16) ? 2 : 4;
        M.out_tma = 0;
        void* out = M.w ? (void*)M.w : M.user;   // fused Muon step: the box is reduce-added into W
        if (P->nsplit == 1 && !M.npack && reinterpret_cast<uintptr_t>(out) % 16 == 0 && (M.ld * esz) % 16 == 0 &&
            ((int64_t)M.n * esz) % 16 == 0) {
            M.out_tma = make_map(enc, mp + kMapEOut, out, M.m, M.n, M.ld * esz, 32, 32, esz == 4 ? F32 : BF,
                                 esz == 4 ? S128 : S64)
                            ? 1
                            : 0;
        }
        const size_t g0 = ph[kGram].size(), s0 = ph[kSquare].size();
        tiles_of(M, i, ph, P->cubic);
        need[2 * i] = (int)(ph[kGram].size() - g0);
        need[2 * i + 1] = (int)(ph[kSquare].size() - s0);
    }
    cudaError_t e = cudaMemcpy(d_mats, mats, sizeof(DevMat) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        *err = std::string("uploading descriptors: ") + cudaGetErrorString(e);
        return PE_ECUDA;
    }
    P->sms = sms;
    P->mat_cost.assign(count, 0.0);
    for (int k = 0; k < 3; ++k) {
        P->ph_t[k].clear();
        P->ph_c[k].clear();
        for (const HostTile& h : ph[k]) {
            P->ph_t[k].push_back(h.t);
            P->ph_c[k].push_back(h.cost);
            P->mat_cost[h.t.mat] += h.cost;
        }
    }
    const size_t ntot = ph[0].size() + ph[1].size() + ph[2].size();
    size_t o = 0;
    char* base = ws;
    auto take = [&](size_t bytes, size_t al) { o = align_up(o, al); char* p = base + o; o += bytes; return p; };
    P->maps = take(sizeof(CUtensorMap) * maps.size(), 1024);
    P->tiles = reinterpret_cast<TileTask*>(take(sizeof(TileTask) * (ntot + 2), 256));
    P->tile_off = reinterpret_cast<int*>(take(sizeof(int) * (sms + 1), 256));
    P->need = reinterpret_cast<int*>(take(sizeof(int) * 2 * count, 256));
    P->need2 = reinterpret_cast<int*>(take(sizeof(int) * 2 * count, 256));
    TileTask* ph_base = reinterpret_cast<TileTask*>(take(sizeof(TileTask) * (ntot + 2), 256));
    size_t ph_pos = 0;
    for (int k = 0; k < 3; ++k) {
        P->ph_tiles[k] = ph_base + ph_pos;
        P->ph_off[k] = reinterpret_cast<int*>(take(sizeof(int) * (sms + 1), 256));
        ph_pos += ph[k].size();
    }
    if (o > ws_bytes) {
        *err = "internal: tcgen05 workspace too small";
        return PE_ECUDA;
    }
    e = cudaMemcpy(P->maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->need, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        *err = std::string("uploading tensor maps: ") + cudaGetErrorString(e);
        return PE_ECUDA;
    }
    if (P->nsplit == 3) P->smem_bytes = (P->bk == 64) ? Cfg<3, 64>::kSmem : Cfg<3, 32>::kSmem;
    else P->smem_bytes = (P->bk == 64) ? Cfg<1, 64>::kSmem : Cfg<1, 32>::kSmem;
    P->smem_bytes2 = Cfg<1, 64, 2>::kSmem;
    P->smem_bytes3 = Cfg<1, 64, 2, 12>::kSmem;
    e = cudaFuncSetAttribute(umma_step_kernel<1, 64, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg<1, 64>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(umma_step_kernel<1, 32, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg<1, 32>::kSmem);
    if (e == cudaSuccess && P->gram_f32)
        e = cudaFuncSetAttribute(umma_step_kernel<1, 64, 0, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg<1, 64>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(umma_step_kernel<3, 64, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg<3, 64>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(umma_step_kernel<3, 32, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg<3, 32>::kSmem);
    if (e != cudaSuccess) {
        *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return PE_ECUDA;
    }
    // 2-SM UMMA: 256 x 256 tiles, needs every padded size to be a multiple of 256
    P->max_clusters2 = 0;
    P->max_clusters3 = 0;
    bool even = (P->nsplit == 1 && P->bk == 64);
    for (int i = 0; i < count && even; ++i) even = (mats[i].sp % 256 == 0) && (mats[i].Lp % 256 == 0);
    if (even) {
        std::vector<int> need2(2 * count, 0);
        for (int k = 0; k < 3; ++k) {
            P->ph2_t[k].clear();
            P->ph2_c[k].clear();
        }
        for (int i = 0; i < count; ++i) {
            const DevMat& M = mats[i];
            const int t2 = M.sp / 256, tl = M.Lp / 256;
            for (int a = 0; a < t2; ++a)
                for (int b = a; b < t2; ++b) {
                    P->ph2_t[kGram].push_back(TileTask{i, a, b, kGram});
                    P->ph2_c[kGram].push_back(256.0 * 256.0 * M.Lp);
                    if (!P->cubic) {
                        P->ph2_t[kSquare].push_back(TileTask{i, a, b, kSquare});
                        P->ph2_c[kSquare].push_back(256.0 * 256.0 * M.sp);
                        need2[2 * i + 1] += 2;
                    }
                    need2[2 * i] += 2;       // each CTA of the pair signals its half
                }
            for (int a = 0; a < t2; ++a)
                for (int b = 0; b < tl; ++b) {
                    P->ph2_t[kApply].push_back(TileTask{i, a, b, kApply});
                    P->ph2_c[kApply].push_back(256.0 * 256.0 * M.sp);
                }
        }
        e = cudaFuncSetAttribute(umma_step_kernel<1, 64, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg<1, 64, 2>::kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(umma_step_kernel<1, 64, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cfg<1, 64, 2>::kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(umma_step_kernel<1, 64, 2, 2, false, 12>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<1, 64, 2, 12>::kSmem);
        if (e == cudaSuccess && P->need2)
            e = cudaMemcpy(P->need2, need2.data(), sizeof(int) * need2.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && P->need2) {
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3(2 * (sms / 2));
            cfg.blockDim = dim3(Cfg<1, 64, 2>::kThreads);
            cfg.dynamicSmemBytes = Cfg<1, 64, 2>::kSmem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, umma_step_kernel<1, 64, 2, 2>, &cfg) == cudaSuccess)
                P->max_clusters2 = std::min(n, sms / 2);
            // the variant with twelve epilogue warps (mode 3)
            cfg.blockDim = dim3(Cfg<1, 64, 2, 12>::kThreads);
            cfg.dynamicSmemBytes = Cfg<1, 64, 2, 12>::kSmem;
            n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, umma_step_kernel<1, 64, 2, 2, false, 12>, &cfg) == cudaSuccess)
                P->max_clusters3 = std::min(n, sms / 2);
        }
        cudaGetLastError();
    }
    if (P->mode != 0 && P->mode != 2 && P->mode != 3) P->mode = 0;
    if (P->mode == 3 && P->max_clusters3 < 1) P->mode = 2;
    if (P->mode == 2 && P->max_clusters2 < 1) P->mode = 0;
    return umma_schedule(P, P->order, err);
}

cudaError_t umma_step(UmmaPlan* P, int t, float a, float b, float c, int last, int phase, int withhold,
                      uint64_t wait_ns, int* status, cudaStream_t st, int* launched) {
    StepArgs A;
    A.nscale = P->nscale;
    A.mats = P->d_mats;
    A.maps = reinterpret_cast<const CUtensorMap*>(P->maps);
    A.need = (P->mode >= 2) ? P->need2 : P->need;
    A.counters = P->counters;
    A.status = status;
    A.a = a;
    A.b = b;
    A.c = c;
    A.step = t;
    A.cur = t & 1;
    A.last = last;
    A.withhold = withhold;
    A.cubic = P->cubic ? 1 : 0;
    A.nmats = P->count;
    A.wait_ns = wait_ns;
    A.prof = reinterpret_cast<long long*>(P->prof);
    *launched = 0;
    auto go = [&](int grid, bool coop) -> cudaError_t {
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3((P->mode == 3) ? Cfg<1, 64, 2, 12>::kThreads : Cfg<1, 64>::kThreads);
        cfg.dynamicSmemBytes = (P->mode == 3) ? P->smem_bytes3 : (P->mode == 2) ? P->smem_bytes2 : P->smem_bytes;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        if (P->mode != 0) {
            // 2-SM pairs; co-residency of the whole grid comes from sizing it
            // by cudaOccupancyMaxActiveClusters at plan time
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
        } else {
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = coop ? 1 : 0;
        }
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ++*launched;
        if (P->nsplit == 3) {
            if (P->bk == 64) return cudaLaunchKernelEx(&cfg, umma_step_kernel<3, 64, 0, 2>, A);
            return cudaLaunchKernelEx(&cfg, umma_step_kernel<3, 32, 0, 2>, A);
        }
        if (P->gram_f32) return cudaLaunchKernelEx(&cfg, umma_step_kernel<1, 64, 0, 2, true>, A);
        if (P->mode == 3) return cudaLaunchKernelEx(&cfg, umma_step_kernel<1, 64, 2, 2, false, 12>, A);
        if (P->mode == 2) {
            if (P->nacc == 2) return cudaLaunchKernelEx(&cfg, umma_step_kernel<1, 64, 2, 2>, A);
            return cudaLaunchKernelEx(&cfg, umma_step_kernel<1, 64, 2, 1>, A);
        }
        if (P->bk == 64) return cudaLaunchKernelEx(&cfg, umma_step_kernel<1, 64, 0, 2>, A);
        return cudaLaunchKernelEx(&cfg, umma_step_kernel<1, 32, 0, 2>, A);
    };
    if (phase < 0) {
        A.off = P->tile_off;
        A.tiles = P->tiles;
        A.dependent = 1;
        return go(P->grid, true);
    }
    A.dependent = 0;
    if (!P->grid_phase[phase]) return cudaSuccess;
    A.off = P->ph_off[phase];
    A.tiles = P->ph_tiles[phase];
    return go(P->grid_phase[phase], false);
}

}  // namespace pe
