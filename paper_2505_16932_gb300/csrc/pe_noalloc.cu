// pe_polar_noalloc: the plain FP32 path of pe_polar for one matrix, with all
// of its device workspace in one fixed, file-scope device array instead of
// memory obtained from cudaMalloc.
//
// Some callers cannot let a library allocate device memory: applications
// whose own allocator takes all of device memory up front (a framework's
// caching pool, an inference server with a fixed memory budget), where a
// library's cudaMalloc either fails or fragments memory the application
// already accounted for; latency-critical loops that must never block on
// the device-wide synchronisation that cudaMalloc and cudaFree can imply;
// and hosts that load this library as a plug-in under a rule that plug-ins
// allocate nothing. For them this entry point uses a static workspace of
// kScratchBytes that exists, on every GPU where the library is loaded, from
// module load until process exit.
//
// In host code the array's name is only a stand-in, not a device address:
// its device address is looked up once per device with cudaGetSymbolAddress
// (the first call on that device) and passed to the kernels. Nothing is
// staged from host memory: a set-up kernel takes the matrix descriptor by
// value and writes it, the task lists and the cleared prepare ticket into
// the array, then the prepare and SIMT kernels of the FP32 path run on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "pe_internal.h"

namespace pe {
namespace {

constexpr size_t kScratchBytes = 32u << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxTiles = 8192;               // prepare + Gram + square + update tiles

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_na_mu;
void* g_na_ptr[kMaxDevices] = {nullptr};

inline int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int na_fail(int code, const std::string& m) {
    set_last_error(m.c_str());
    return code;
}

// Writes the descriptor M to *d_mat, the task lists to `t` (prepare strips,
// then the Gram and square tiles on and above the diagonal, then the update
// tiles, in the order of the host loops of pe_polar's FP32 plan) and clears
// the 64-byte ticket / status block. One block; thread k takes rows k,
// k + blockDim, ... of each list.
__global__ void na_setup_kernel(DevMat M, DevMat* d_mat, TileTask* t, int nb, int ts, int tl, unsigned* ticket) {
    if (threadIdx.x == 0) *d_mat = M;
    if (threadIdx.x < 16) ticket[threadIdx.x] = 0u;
    const int rows_p = M.sp / kPrepRows;
    const int n_prep = rows_p * nb;
    const int n_sym = ts * (ts + 1) / 2;
    for (int a = threadIdx.x; a < rows_p; a += blockDim.x)
        for (int b = 0; b < nb; ++b) t[a * nb + b] = TileTask{0, a, b, -1};
    for (int a = threadIdx.x; a < ts; a += blockDim.x) {
        const int row0 = a * ts - a * (a - 1) / 2;   // tiles (a', b), a' < a, b >= a'
        for (int b = a; b < ts; ++b) {
            t[n_prep + row0 + (b - a)] = TileTask{0, a, b, kGram};
            t[n_prep + n_sym + row0 + (b - a)] = TileTask{0, a, b, kSquare};
        }
    }
    for (int a = threadIdx.x; a < ts; a += blockDim.x)
        for (int b = 0; b < tl; ++b) t[n_prep + 2 * n_sym + a * tl + b] = TileTask{0, a, b, kApply};
}

}  // namespace
}  // namespace pe

extern "C" int pe_polar_noalloc(void* X, int64_t m, int64_t n, const double* table, int T, void* stream) {
    using namespace pe;
    if (!X) return na_fail(PE_EINVAL, "X is NULL");
    if (m < 1 || n < 1) return na_fail(PE_EINVAL, "sizes must be >= 1");
    if (!table) return na_fail(PE_EINVAL, "table is NULL");
    if (T < 1 || T > kMaxSteps) return na_fail(PE_EINVAL, "T must be in 1..64");
    if (reinterpret_cast<uintptr_t>(X) % 4) return na_fail(PE_EINVAL, "misaligned matrix pointer");
    for (int i = 0; i < 3 * T; ++i)
        if (!std::isfinite(table[i])) return na_fail(PE_EINVAL, "non-finite coefficient in table");
    if (m > (1 << 20) || n > (1 << 20)) return na_fail(PE_EINVAL, "matrix too large");
    const int64_t s = std::min(m, n), L = std::max(m, n);
    const int64_t sp = rup(s, kPadS), Lp = rup(L, kPadL);
    // workspace layout: [descriptor | tasks | partials | scale | ticket | X | X' | A | B]
    const int64_t nb = (Lp + kPrepCols - 1) / kPrepCols;
    const int64_t n_prep = (sp / kPrepRows) * nb;
    const int64_t ts = sp / 128, tl = Lp / 128;
    const int64_t n_sym = ts * (ts + 1) / 2, n_app = ts * tl;
    const int64_t n_tasks = n_prep + 2 * n_sym + n_app;
    size_t off = 0;
    auto take = [&](size_t bytes, size_t al) { off = (off + al - 1) / al * al; size_t o = off; off += bytes; return o; };
    const size_t o_mat = take(sizeof(DevMat), 256);
    const size_t o_tasks = take(sizeof(TileTask) * (size_t)n_tasks, 256);
    const size_t o_part = take(sizeof(double) * (size_t)n_prep, 256);
    const size_t o_scale = take(sizeof(float), 256);
    const size_t o_ticket = take(64, 256);
    const size_t o_xf = take(4 * (size_t)(sp * Lp), 256);
    const size_t o_xf2 = take(4 * (size_t)(sp * Lp), 256);
    const size_t o_af = take(4 * (size_t)(sp * sp), 256);
    const size_t o_bf = take(4 * (size_t)(sp * sp), 256);
    if (off > kScratchBytes || n_tasks > kMaxTiles)
        return na_fail(PE_EINVAL, "matrix needs " + std::to_string(off) + " bytes of workspace; the static "
                                  "workspace of pe_polar_noalloc holds " + std::to_string(kScratchBytes));

    std::lock_guard<std::mutex> lk(g_na_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(PE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(PE_EUNSUPPORTED, "device index out of range");
    if (!g_na_ptr[dev]) {
        // set-up, once per device (this device is current): the array's
        // device address
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(PE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = p;
    }
    char* base = static_cast<char*>(g_na_ptr[dev]);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    DevMat M;
    memset(&M, 0, sizeof(M));
    M.user = X;
    M.ld = n;
    M.m = (int32_t)m;
    M.n = (int32_t)n;
    M.trans = m > n;
    M.io = PE_IO_FP32;
    M.s = (int32_t)s;
    M.L = (int32_t)L;
    M.sp = (int32_t)sp;
    M.Lp = (int32_t)Lp;
    M.part0 = 0;
    M.npart = (int32_t)n_prep;
    M.xf = reinterpret_cast<float*>(base + o_xf);
    M.xf2 = reinterpret_cast<float*>(base + o_xf2);
    M.af = reinterpret_cast<float*>(base + o_af);
    M.bfp = reinterpret_cast<float*>(base + o_bf);

    DevMat* d_mat = reinterpret_cast<DevMat*>(base + o_mat);
    TileTask* d_tasks = reinterpret_cast<TileTask*>(base + o_tasks);
    double* d_part = reinterpret_cast<double*>(base + o_part);
    float* d_scale = reinterpret_cast<float*>(base + o_scale);
    unsigned* d_ticket = reinterpret_cast<unsigned*>(base + o_ticket);
    int* d_status = reinterpret_cast<int*>(base + o_ticket + 16);
    const int g0 = (int)n_prep, q0 = (int)(n_prep + n_sym), a0 = (int)(n_prep + 2 * n_sym);
    // the previous call's contents stay in the array: the set-up kernel
    // rewrites the descriptor and task lists and clears the ticket and status
    na_setup_kernel<<<1, 256, 0, st>>>(M, d_mat, d_tasks, (int)nb, (int)ts, (int)tl, d_ticket);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_prepare(d_mat, 1, d_tasks, (int)n_prep, d_part, 1.01f, 1e-7f, kPrepF32, d_scale, d_status,
                           d_status + 1, 0, d_ticket, st);
    for (int step = 0; step < T && e == cudaSuccess; ++step) {
        const float a = (float)table[3 * step], b = (float)table[3 * step + 1], c = (float)table[3 * step + 2];
        const int last = (step == T - 1);
        e = launch_simt_phase(d_mat, d_tasks + g0, q0 - g0, kGram, a, b, c, step & 1, last, step == 0, d_scale, st);
        if (e == cudaSuccess)
            e = launch_simt_phase(d_mat, d_tasks + q0, a0 - q0, kSquare, a, b, c, step & 1, last, step == 0, d_scale,
                                  st);
        if (e == cudaSuccess)
            e = launch_simt_phase(d_mat, d_tasks + a0, (int)n_tasks - a0, kApply, a, b, c, step & 1, last,
                                  step == 0, d_scale, st);
    }
    if (e != cudaSuccess) return na_fail(PE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return PE_OK;
}
