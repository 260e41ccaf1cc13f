// tcgen05 (UMMA) path of the online stage: BF16 and split-BF16 (BF16x3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pe_internal.h"

namespace pe {

// Host-side plan of the persistent grouped step kernel.
struct UmmaPlan {
    int count = 0;
    int dtype = 0;
    int nsplit = 1;          // 1 (BF16) or 3 (BF16x3)
    int grid = 0;            // persistent CTAs (<= SMs)
    int grid_phase[3] = {0, 0, 0};
    void* maps = nullptr;    // device array of CUtensorMap, kMapsPerMat per matrix
    int* tile_off = nullptr; // device CSR offsets per CTA (grid + 1), fused schedule
    TileTask* tiles = nullptr;
    int ntiles = 0;
    int* ph_off[3] = {nullptr, nullptr, nullptr};  // per-phase schedules (phased mode)
    TileTask* ph_tiles[3] = {nullptr, nullptr, nullptr};
    int* need = nullptr;     // device: per matrix [n_gram, n_square]
    int* counters = nullptr; // device: per matrix [gram_done, square_done]
    const DevMat* d_mats = nullptr;
    size_t smem_bytes = 0;
    int apply_bn = 256;
    int bk = 64;             // k-block of the tcgen05 kernel (64 or 32)
    int order = 0;           // tile order (see umma_schedule)
    int mode = 0;            // 0 one CTA per 128x256 tile; 2 2-SM UMMA (cta_group::2) on
                             // 256x256 tiles; 3 the same with twelve epilogue warps and
                             // four operand stages (instead of eight and five)
    int nacc = 2;            // accumulators per CTA in mode 2 (1 or 2)
    bool cubic = false;      // every step has c = 0 (BF16 only): B = b A comes from the
                             // Gram epilogue and there are no square tiles
    bool gram_f32 = false;   // long-side split: the Gram writes the full FP32 A into DevMat::af
                             // (its own kernel instantiation; mode 0, 64-wide k-blocks)
    int max_clusters2 = 0;   // co-resident clusters of two, 2-SM kernel (0: unavailable)
    size_t smem_bytes2 = 0;  // dynamic shared memory of the 2-SM kernel
    int max_clusters3 = 0;   // the same for the mode-3 kernel
    size_t smem_bytes3 = 0;
    int* need2 = nullptr;    // device: per matrix readiness targets of 2-SM plans
    std::vector<TileTask> ph2_t[3];   // 256 x 256 tiles (2-SM plans)
    std::vector<double> ph2_c[3];
    void* prof = nullptr;    // optional device buffer of 32 int64 per CTA (debug)
    const float* nscale = nullptr;   // device: per-matrix normalisation factors
    // host copy of the per-phase tiles and their costs (for re-scheduling)
    int sms = 0;
    std::vector<TileTask> ph_t[3];
    std::vector<double> ph_c[3];
    std::vector<double> mat_cost;
};

size_t umma_workspace_bytes(const DevMat* mats, int count);

// Builds tensor maps and schedules inside `ws` (device memory of
// umma_workspace_bytes()); sets DevMat::out_tma and re-uploads the
// descriptors to d_mats.
int umma_build(UmmaPlan* P, DevMat* mats, DevMat* d_mats, int count, int dtype, int sms,
               char* ws, size_t ws_bytes, int* counters, bool tune, std::string* err);

// Rebuilds and uploads the fused and phased tile schedules for a tile order
// (0 longest-first, 1 column-grouped raster).
int umma_schedule(UmmaPlan* P, int order, std::string* err);

// Enqueue polynomial step t (0-based). phase < 0: one persistent launch of
// the whole step with per-matrix readiness waits; phase 0/1/2: one grouped
// launch of that product only (Gram, square, update).
cudaError_t umma_step(UmmaPlan* P, int t, float a, float b, float c, int last, int phase,
                      int withhold, uint64_t wait_ns, int* status, cudaStream_t st, int* launched);

}  // namespace pe
