// C ABI of the library: argument checks, workspace, cached plans (grouped
// task lists, tensor maps, captured CUDA graphs) and the launch sequence of
// the online stage (Alg. 1, online box):
//   prepare (one pass: cast + transpose + pad + Frobenius norm partials, last
//   block computes the normalisation factors)  ->  T x [Gram -> A^2 -> update]
//   (the first step applies the normalisation factor)
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pe_internal.h"
#include "pe_umma.h"

namespace pe {
namespace {

thread_local std::string g_err;
std::mutex g_mu;
std::atomic<int64_t> g_launches{0};
int64_t g_dbg_withhold = -1;
int64_t g_dbg_wait_ns = 0;
bool g_dbg_fail_alloc = false;
void* g_dbg_prof = nullptr;
int g_dbg_bk = 0;      // 0: default k-block
int g_dbg_order = -1;  // -1: default tile order
int g_dbg_mode = -1;   // -1: autotuned; 0 / 2: force the tcgen05 kernel mode
int g_dbg_nacc = 0;    // 0: default accumulators of 2-SM plans; 1 or 2
bool g_dbg_nopair = false;   // true: no packing of small matrices in plans built from now on

// tracing: (kind, start, stop) event triples recorded on the call's stream
struct TraceRec { int kind; cudaEvent_t a, b; };
bool g_trace = false;
std::vector<TraceRec> g_trace_recs;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t trace_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct TraceScope {
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    TraceScope(int k, cudaStream_t s) : kind(k), st(s) {
        if (g_trace) {
            a = trace_event();
            cudaEventRecord(a, st);
        }
    }
    ~TraceScope() {
        if (a) {
            cudaEvent_t b = trace_event();
            cudaEventRecord(b, st);
            g_trace_recs.push_back(TraceRec{kind, a, b});
        }
    }
};

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return PE_ECUDA;
}

#define PE_CU(call)                                   \
    do {                                              \
        cudaError_t _e = (call);                      \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct DeviceState {
    bool init = false;
    int sms = 0, major = 0, minor = 0;
    int* status = nullptr;   // device status word (bit 0 timeout, bit 1 non-finite norm)
    cudaStream_t cap = nullptr;  // private stream used to capture plans
};
std::vector<DeviceState> g_dev;

int device_state(DeviceState** out) {
    int dev = 0;
    PE_CU(cudaGetDevice(&dev));
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DeviceState& d = g_dev[dev];
    if (!d.init) {
        PE_CU(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        PE_CU(cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev));
        PE_CU(cudaDeviceGetAttribute(&d.minor, cudaDevAttrComputeCapabilityMinor, dev));
        PE_CU(cudaMalloc(&d.status, 64));
        PE_CU(cudaMemset(d.status, 0, 64));
        PE_CU(cudaStreamCreateWithFlags(&d.cap, cudaStreamNonBlocking));
        d.init = true;
    }
    *out = &d;
    return PE_OK;
}

// ------------------------------------------------------------------ plans

// FP32 path: Gram reductions longer than this run in chunks (see pe_simt.cu)
constexpr int64_t kGramChunk = 4096;
constexpr int kMaxGramChunks = 256;

// internal plan flags (above the public PE_BATCH_* bits)
constexpr unsigned kFlagSplit = 1u << 16;           // long-side split plan (pe_split_*)
constexpr unsigned kFlagSplitShortCols = 1u << 17;  // split plan whose shared short side is the columns

struct PlanKey {
    int dev, dtype, T, io, count;
    unsigned flags;
    float scale, eps;
    std::vector<uintptr_t> ptrs;
    std::vector<int64_t> dims;   // m, n, ld per matrix
    std::vector<float> coef;     // 3*T
    // fused Muon step: momentum and weight buffers per matrix (empty otherwise)
    std::vector<uintptr_t> mom, w;
    float beta = 0.f, lr = 0.f;
    // Alg. 4 (fast rectangular iteration): steps per restart block (0: the
    // ordinary iteration) and the first block's shift of Y
    int restart = 0;
    float shift = 0.f;
    bool operator==(const PlanKey& o) const {
        return dev == o.dev && dtype == o.dtype && T == o.T && io == o.io && count == o.count &&
               flags == o.flags && scale == o.scale && eps == o.eps && ptrs == o.ptrs &&
               dims == o.dims && coef == o.coef && mom == o.mom && w == o.w && beta == o.beta && lr == o.lr &&
               restart == o.restart && shift == o.shift;
    }
};

struct Plan {
    PlanKey key;
    DeviceState* ds = nullptr;
    std::vector<DevMat> mats;
    char* ws = nullptr;           // one allocation: descriptors, task lists, buffers
    size_t ws_bytes = 0;
    DevMat* d_mats = nullptr;
    double* d_partials = nullptr; // one per prepare tile
    float* d_nscale = nullptr;    // per-matrix 1 / (scale ||G||_F + eps)
    unsigned* d_ticket = nullptr; // prepare's last-block ticket
    TileTask* d_prep = nullptr;
    int n_prep = 0;
    TileTask* d_tiles[3] = {nullptr, nullptr, nullptr};   // SIMT per-phase lists
    int n_tiles[3] = {0, 0, 0};
    TileTask* d_red = nullptr;    // SIMT: tiles of split Grams (partials summed by the reduce launch)
    int n_red = 0;
    // Alg. 4 plans: task lists of the block's s x s products and of their
    // split-K reductions (see enqueue_fast)
    enum { kFSq0, kFSq1, kFP0, kFP1, kFR0, kFR1, kFH, kFQ0, kFQ1, kFLists };
    GemmTask* d_fast[kFLists] = {};
    int n_fast[kFLists] = {};
    FastReduce* d_fred[kFLists] = {};
    int n_fred[kFLists] = {};
    int* d_counters = nullptr;
    int n_counters = 0;
    UmmaPlan umma;                // tcgen05 path (tensor maps, persistent schedule)
    cudaGraphExec_t exec = nullptr;
    int kernels_per_run = 0;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (ws) cudaFree(ws);
    }
};

std::list<std::unique_ptr<Plan>> g_plans;   // most recently used first
constexpr size_t kMaxPlans = 16;

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes, size_t align = 1024) {
        off = round_up(off, align);
        size_t o = off;
        off += bytes;
        return o;
    }
};

int build_plan(const PlanKey& key, Plan** out) {
    auto P = std::make_unique<Plan>();
    P->key = key;
    PE_CU(cudaGetDevice(&P->key.dev));
    int st = device_state(&P->ds);
    if (st != PE_OK) return st;
    if (!(P->ds->major == 10 && P->ds->minor == 3))
        return fail(PE_EUNSUPPORTED, "this library is built for sm_103 (GB300) only");

    const int dtype = key.dtype;
    // Descriptors: one per matrix, except that on the BF16 path matrices with
    // a short side <= 64 of one shape are packed, up to kMaxPack, into a
    // descriptor of kMaxPack 64-row blocks (block k holds matrix k's canonical
    // rows), and the Gram keeps the diagonal 64 x 64 blocks only, so A,
    // B = b A + c A^2 and the update stay block diagonal: the pack fills the
    // MMA tiles that each such matrix alone would pad, and a pack's 256 rows
    // keep the plan eligible for the 2-SM kernel. A shape seen once is not
    // packed.
    std::vector<std::vector<int>> src;   // per descriptor: its matrices
    {
        const bool can_pack = dtype == PE_BF16 && key.w.empty() && !(key.flags & kFlagSplit) && !g_dbg_nopair;
        std::map<std::pair<int64_t, int64_t>, int> shape_n;
        if (can_pack)
            for (int i = 0; i < key.count; ++i) {
                const int64_t m = key.dims[3 * i], n = key.dims[3 * i + 1];
                if (std::min(m, n) <= 64 && key.dims[3 * i + 2] == n) ++shape_n[{m, n}];
            }
        std::map<std::pair<int64_t, int64_t>, int> open;   // shape -> descriptor with room
        for (int i = 0; i < key.count; ++i) {
            const int64_t m = key.dims[3 * i], n = key.dims[3 * i + 1];
            auto sn = shape_n.find({m, n});
            if (sn != shape_n.end() && sn->second >= 2 && key.dims[3 * i + 2] == n) {
                auto it = open.find({m, n});
                if (it != open.end()) {
                    src[it->second].push_back(i);
                    if ((int)src[it->second].size() == kMaxPack) open.erase(it);
                    continue;
                }
                open[{m, n}] = (int)src.size();
            }
            src.push_back({i});
        }
        // a descriptor opened for packing keeps its kMaxPack blocks even if
        // fewer matrices arrived (the missing blocks are padding)
        for (auto& d : src)
            if (d.size() == 1) {
                const int64_t m = key.dims[3 * d[0]], n = key.dims[3 * d[0] + 1];
                auto sn = shape_n.find({m, n});
                if (sn != shape_n.end() && sn->second >= 2) d.push_back(-1);   // marks a pack of one
            }
    }
    const int count = (int)src.size();
    P->mats.resize(count);
    Carve cv;
    // layout of the single workspace allocation
    const size_t o_mats = cv.take(sizeof(DevMat) * count, 64);
    std::vector<TileTask> prep, tl[3], red;
    struct Off { size_t xf, xf2, xh0, xh1, xl0, xl1, xq, af, ah, al, bfp, bh, bl, gpart, btr, fq, fp, fr, fh; };
    std::vector<Off> offs(count);
    int part = 0;
    for (int i = 0; i < count; ++i) {
        DevMat& M = P->mats[i];
        memset(&M, 0, sizeof(M));
        const int u = src[i][0];
        const int64_t m = key.dims[3 * u], n = key.dims[3 * u + 1], ld = key.dims[3 * u + 2];
        M.user = reinterpret_cast<void*>(key.ptrs[u]);
        if (src[i].size() > 1) {   // a pack
            M.npack = 1;
            for (size_t k = 1; k < src[i].size(); ++k)
                if (src[i][k] >= 0) M.pack[M.npack++ - 1] = reinterpret_cast<void*>(key.ptrs[src[i][k]]);
        }
        if (!key.w.empty()) {
            M.mom = reinterpret_cast<float*>(key.mom[u]);
            M.w = reinterpret_cast<float*>(key.w[u]);
            M.beta = key.beta;
            M.lr = key.lr;
        }
        M.ld = ld;
        M.m = (int32_t)m;
        M.n = (int32_t)n;
        M.trans = m > n;
        M.io = key.io;
        M.s = (int32_t)std::min(m, n);
        M.L = (int32_t)std::max(m, n);
        if (key.flags & kFlagSplit) {
            // long-side split: the shared short side is fixed by the caller,
            // the local long extent may be the smaller one
            M.trans = (key.flags & kFlagSplitShortCols) ? 1 : 0;
            M.s = (int32_t)(M.trans ? n : m);
            M.L = (int32_t)(M.trans ? m : n);
        }
        M.sp = (int32_t)round_up(M.s, kPadS);
        if (M.npack) M.sp = 64 * kMaxPack;
        M.Lp = (int32_t)round_up(M.L, kPadL);
        M.part0 = part;
        for (int a = 0; a < M.sp / kPrepRows; ++a)
            for (int b = 0; b < (M.Lp + kPrepCols - 1) / kPrepCols; ++b) {
                prep.push_back(TileTask{i, a, b, -1});
                ++part;
            }
        M.npart = part - M.part0;
        if (M.npack) M.npart /= kMaxPack;   // per 64-row block
        const size_t sL = (size_t)M.sp * M.Lp, ss = (size_t)M.sp * M.sp;
        Off& o = offs[i];
        memset(&o, 0, sizeof(o));
        if (dtype == PE_FP32) {
            o.xf = cv.take(4 * sL);
            o.xf2 = cv.take(4 * sL);
            o.af = cv.take(4 * ss);
            o.bfp = cv.take(4 * ss);
            // Gram reductions longer than kGramChunk run as chunks of at most
            // kGramChunk columns (at most kMaxGramChunks of them, and at most
            // 1 GiB of partial Grams per matrix)
            int ks = 1;
            if (!(key.flags & kFlagSplit) && M.Lp > kGramChunk) {
                ks = (int)std::min<int64_t>((M.Lp + kGramChunk - 1) / kGramChunk, kMaxGramChunks);
                while (ks > 1 && (size_t)ks * 4 * ss > ((size_t)1 << 30)) --ks;
            }
            const int64_t chunk = round_up((M.Lp + ks - 1) / ks, 16);
            M.ksplit = (int32_t)((M.Lp + chunk - 1) / chunk);
            M.kchunk = (int32_t)chunk;
            if (M.ksplit > 1) o.gpart = cv.take(4 * ss * (size_t)M.ksplit);
            if (key.restart > 0) {   // Alg. 4: Q (second buffer), P, R, H
                o.fq = cv.take(4 * ss);
                o.fp = cv.take(4 * ss);
                o.fr = cv.take(4 * ss);
                o.fh = cv.take(4 * ss);
            }
        } else {
            o.xh0 = cv.take(2 * sL);
            o.xh1 = cv.take(2 * sL);
            o.ah = cv.take(2 * ss);
            o.bh = cv.take(2 * ss);
            if (dtype == PE_BF16) o.xq = cv.take(sL);
            if (dtype == PE_BF16) o.btr = cv.take(4 * (size_t)(M.sp / 32), 64);   // tr(A) parts
            if (dtype == PE_BF16 && (key.flags & kFlagSplit)) o.af = cv.take(4 * ss);   // partial Gram, FP32
            if (dtype == PE_BF16X3) {
                o.xf = cv.take(4 * sL);
                o.af = cv.take(4 * ss);
                o.xl0 = cv.take(2 * sL);
                o.xl1 = cv.take(2 * sL);
                o.al = cv.take(2 * ss);
                o.bl = cv.take(2 * ss);
            }
        }
        if (dtype == PE_FP32) {
            const int ts = M.sp / 128, tL = M.Lp / 128;
            for (int a = 0; a < ts; ++a)
                for (int b = a; b < ts; ++b) {
                    if (M.ksplit > 1) {
                        for (int k = 0; k < M.ksplit; ++k) tl[kGram].push_back(TileTask{i, a, b, kGram | (k << 8)});
                        red.push_back(TileTask{i, a, b, kGram});
                    } else {
                        tl[kGram].push_back(TileTask{i, a, b, kGram});
                    }
                    tl[kSquare].push_back(TileTask{i, a, b, kSquare});
                }
            for (int a = 0; a < ts; ++a)
                for (int b = 0; b < tL; ++b) tl[kApply].push_back(TileTask{i, a, b, kApply});
        }
    }
    P->n_prep = (int)prep.size();
    const size_t o_part = cv.take(sizeof(double) * prep.size(), 64);
    const size_t o_nscale = cv.take(sizeof(float) * kMaxPack * count, 64);   // per descriptor and block
    const size_t o_ticket = cv.take(sizeof(unsigned) * kMaxPack * count, 64);   // prepare: per descriptor and block
    const size_t o_prep = cv.take(sizeof(TileTask) * prep.size(), 64);
    size_t o_tl[3];
    for (int k = 0; k < 3; ++k) {
        P->n_tiles[k] = (int)tl[k].size();
        o_tl[k] = cv.take(sizeof(TileTask) * std::max<size_t>(1, tl[k].size()), 64);
    }
    P->n_red = (int)red.size();
    const size_t o_red = cv.take(sizeof(TileTask) * std::max<size_t>(1, red.size()), 64);
    // Alg. 4: products with few output tiles are split along K (about two
    // waves of blocks per launch; chunks of at least 128): the split factor
    // of matrix i in a list is min(ks_list, sp_i / 128); symmetric outputs
    // (Sq, R, H) are computed on their upper tiles
    size_t o_fast[Plan::kFLists] = {}, o_fred[Plan::kFLists] = {};
    std::vector<size_t> o_fpart(count, 0);
    int ks_list[2] = {1, 1};   // [full, symmetric] products
    auto fast_ks = [&](int i, bool sym) { return std::max(1, std::min(ks_list[sym ? 1 : 0], P->mats[i].sp / 128)); };
    size_t fast_tasks = 0;
    if (key.restart > 0) {
        size_t nfull = 0, nsym = 0;
        for (int i = 0; i < count; ++i) {
            const size_t nt = (size_t)P->mats[i].sp / 128;
            nfull += nt * nt;
            nsym += nt * (nt + 1) / 2;
        }
        const size_t want = 2 * (size_t)std::max(1, P->ds->sms);
        ks_list[0] = (int)std::min<size_t>(8, std::max<size_t>(1, (want + nfull - 1) / nfull));
        ks_list[1] = (int)std::min<size_t>(8, std::max<size_t>(1, (want + nsym - 1) / nsym));
        for (int i = 0; i < count; ++i) {
            const size_t nt = (size_t)P->mats[i].sp / 128;
            fast_tasks += nt * nt * (size_t)std::max(fast_ks(i, false), fast_ks(i, true));
            const int ksm = std::max(fast_ks(i, false), fast_ks(i, true));
            if (ksm > 1) o_fpart[i] = cv.take(sizeof(float) * (size_t)ksm * P->mats[i].sp * P->mats[i].sp);
        }
        for (int k = 0; k < Plan::kFLists; ++k) {
            o_fast[k] = cv.take(sizeof(GemmTask) * fast_tasks, 64);
            o_fred[k] = cv.take(sizeof(FastReduce) * std::max<size_t>(1, fast_tasks), 64);
        }
    }
    P->n_counters = 2 * count + 64;
    const size_t o_cnt = cv.take(sizeof(int) * P->n_counters, 64);
    size_t o_umma = 0, umma_bytes = 0;
    if (dtype != PE_FP32) {
        umma_bytes = umma_workspace_bytes(P->mats.data(), count);
        o_umma = cv.take(umma_bytes, 1024);
    }
    P->ws_bytes = cv.off;
    if (g_dbg_fail_alloc) {
        g_dbg_fail_alloc = false;
        return fail(PE_ENOMEM, "workspace allocation failed (injected)");
    }
    cudaError_t e = cudaMalloc(&P->ws, P->ws_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        P->ws = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? PE_ENOMEM : PE_ECUDA,
                    std::string("workspace allocation of ") + std::to_string(P->ws_bytes) +
                        " bytes failed: " + cudaGetErrorString(e));
    }
    char* base = P->ws;
    for (int i = 0; i < count; ++i) {
        DevMat& M = P->mats[i];
        const Off& o = offs[i];
        if (dtype == PE_FP32) {
            M.xf = reinterpret_cast<float*>(base + o.xf);
            M.xf2 = reinterpret_cast<float*>(base + o.xf2);
            M.af = reinterpret_cast<float*>(base + o.af);
            M.bfp = reinterpret_cast<float*>(base + o.bfp);
            if (M.ksplit > 1) M.gpart = reinterpret_cast<float*>(base + o.gpart);
        } else {
            M.xh[0] = reinterpret_cast<bf16*>(base + o.xh0);
            M.xh[1] = reinterpret_cast<bf16*>(base + o.xh1);
            M.ah = reinterpret_cast<bf16*>(base + o.ah);
            M.bh = reinterpret_cast<bf16*>(base + o.bh);
            if (dtype == PE_BF16) M.xq = reinterpret_cast<int8_t*>(base + o.xq);
            if (dtype == PE_BF16) M.btr = reinterpret_cast<float*>(base + o.btr);
            if (dtype == PE_BF16 && (key.flags & kFlagSplit)) M.af = reinterpret_cast<float*>(base + o.af);
            if (dtype == PE_BF16X3) {
                M.xf = reinterpret_cast<float*>(base + o.xf);
                M.af = reinterpret_cast<float*>(base + o.af);
                M.xl[0] = reinterpret_cast<bf16*>(base + o.xl0);
                M.xl[1] = reinterpret_cast<bf16*>(base + o.xl1);
                M.al = reinterpret_cast<bf16*>(base + o.al);
                M.bl = reinterpret_cast<bf16*>(base + o.bl);
            }
        }
    }
    P->d_mats = reinterpret_cast<DevMat*>(base + o_mats);
    P->d_partials = reinterpret_cast<double*>(base + o_part);
    P->d_nscale = reinterpret_cast<float*>(base + o_nscale);
    P->d_ticket = reinterpret_cast<unsigned*>(base + o_ticket);
    P->d_prep = reinterpret_cast<TileTask*>(base + o_prep);
    for (int k = 0; k < 3; ++k) P->d_tiles[k] = reinterpret_cast<TileTask*>(base + o_tl[k]);
    P->d_red = reinterpret_cast<TileTask*>(base + o_red);
    std::vector<GemmTask> fast_lists[Plan::kFLists];
    std::vector<FastReduce> fred_lists[Plan::kFLists];
    if (key.restart > 0) {
        // Alg. 4 task lists. Q alternates between B (bfp, read by the update
        // kernel) and fq: Q_j of a k-step block lies in Qb[(k - j) & 1], so Q_k
        // lands in bfp. Lists by the buffer that holds the previous Q (p):
        //   Sq[p]  Q_1 = a I + b Y + c Y Y into Qb[p]
        //   P[p]   P = Y Qb[p]          R[p]  R = Qb[p]^T P
        //   H      H = a I + b R + c R R  Q[p]  Qb[p ^ 1] = Qb[p] H
        std::vector<GemmTask> lists[Plan::kFLists];
        for (int i = 0; i < count; ++i) {
            const DevMat& M = P->mats[i];
            const Off& o = offs[i];
            float* Y = reinterpret_cast<float*>(base + o.af);
            float* Qb[2] = {reinterpret_cast<float*>(base + o.bfp), reinterpret_cast<float*>(base + o.fq)};
            float* Pm = reinterpret_cast<float*>(base + o.fp);
            float* R = reinterpret_cast<float*>(base + o.fr);
            float* H = reinterpret_cast<float*>(base + o.fh);
            const int sp = M.sp, nt = sp / 128;
            float* part = o_fpart[i] ? reinterpret_cast<float*>(base + o_fpart[i]) : nullptr;
            auto add = [&](int list, const float* a, const float* b, const float* e, float* c, bool sym) {
                const int ks = fast_ks(i, sym);
                const int chunk = (int)round_up((sp + ks - 1) / ks, 16);
                const int nks = (sp + chunk - 1) / chunk;
                for (int tm = 0; tm < nt; ++tm)
                    for (int tn = sym ? tm : 0; tn < nt; ++tn) {
                        if (nks == 1) {
                            lists[list].push_back(
                                GemmTask{a, b, e, c, sp, sp, sp, sp, 0, sp, tm, tn, sym ? kGemmMirror : 0, 0});
                            continue;
                        }
                        for (int k = 0; k < nks; ++k)
                            lists[list].push_back(GemmTask{a, b, nullptr, part + (size_t)k * sp * sp, sp, sp, sp, sp,
                                                           k * chunk, std::min(chunk, sp - k * chunk), tm, tn,
                                                           kGemmPartial, 0});
                        fred_lists[list].push_back(
                            FastReduce{part, e, c, (int64_t)sp * sp, nks, sp, tm, tn, sym ? kGemmMirror : 0, 0});
                    }
            };
            for (int p = 0; p < 2; ++p) {
                add(Plan::kFSq0 + p, Y, Y, Y, Qb[p], true);
                add(Plan::kFP0 + p, Y, Qb[p], nullptr, Pm, false);
                add(Plan::kFR0 + p, Qb[p], Pm, nullptr, R, true);
                add(Plan::kFQ0 + p, Qb[p], H, nullptr, Qb[p ^ 1], false);
            }
            add(Plan::kFH, R, R, R, H, true);
        }
        for (int k = 0; k < Plan::kFLists; ++k) {
            P->d_fast[k] = reinterpret_cast<GemmTask*>(base + o_fast[k]);
            P->n_fast[k] = (int)lists[k].size();
            P->d_fred[k] = reinterpret_cast<FastReduce*>(base + o_fred[k]);
            P->n_fred[k] = (int)fred_lists[k].size();
            fast_lists[k].swap(lists[k]);   // uploaded after the workspace is zeroed
        }
    }
    P->d_counters = reinterpret_cast<int*>(base + o_cnt);
    // zero the whole workspace once: the padding of every canonical buffer
    // stays zero from here on (prepare skips strips of padding rows), and the
    // tickets and counters start at zero
    PE_CU(cudaMemset(P->ws, 0, P->ws_bytes));
    for (int i = 0; i < count; ++i)
        if (P->mats[i].xq) PE_CU(cudaMemset(P->mats[i].xq, 0x80, (size_t)P->mats[i].sp * P->mats[i].Lp));   // code of 0
    PE_CU(cudaMemcpy(P->d_mats, P->mats.data(), sizeof(DevMat) * count, cudaMemcpyHostToDevice));

    PE_CU(cudaMemcpy(P->d_prep, prep.data(), sizeof(TileTask) * prep.size(), cudaMemcpyHostToDevice));
    for (int k = 0; k < 3; ++k)
        if (!tl[k].empty())
            PE_CU(cudaMemcpy(P->d_tiles[k], tl[k].data(), sizeof(TileTask) * tl[k].size(),
                             cudaMemcpyHostToDevice));
    if (!red.empty())
        PE_CU(cudaMemcpy(P->d_red, red.data(), sizeof(TileTask) * red.size(), cudaMemcpyHostToDevice));
    for (int k = 0; k < Plan::kFLists; ++k) {
        if (!fast_lists[k].empty())
            PE_CU(cudaMemcpy(P->d_fast[k], fast_lists[k].data(), sizeof(GemmTask) * fast_lists[k].size(),
                             cudaMemcpyHostToDevice));
        if (!fred_lists[k].empty())
            PE_CU(cudaMemcpy(P->d_fred[k], fred_lists[k].data(), sizeof(FastReduce) * fred_lists[k].size(),
                             cudaMemcpyHostToDevice));
    }
    PE_CU(cudaMemset(P->d_counters, 0, sizeof(int) * P->n_counters));
    if (dtype != PE_FP32) {
        const bool tune = false;   // schedules are tuned after the plan is cached (autotune)
        P->umma.nscale = P->d_nscale;
        if (g_dbg_bk == 32 || g_dbg_bk == 64) P->umma.bk = g_dbg_bk;
        if (g_dbg_order >= 0) P->umma.order = g_dbg_order;
        if (g_dbg_mode >= 0) P->umma.mode = g_dbg_mode;
        if (g_dbg_nacc == 1 || g_dbg_nacc == 2) P->umma.nacc = g_dbg_nacc;
        // degree-3 tables (c = 0 in every step) skip the square phase on the BF16 path
        bool cubic = (dtype == PE_BF16) && !(key.flags & kFlagSplit);   // the split exchanges A itself
        P->umma.gram_f32 = (key.flags & kFlagSplit) != 0;
        if (P->umma.gram_f32) {
            P->umma.mode = 0;
            P->umma.bk = 64;
        }
        for (int t = 0; t < key.T && cubic; ++t) cubic = (key.coef[3 * t + 2] == 0.f);
        P->umma.cubic = cubic;
        int ust = umma_build(&P->umma, P->mats.data(), P->d_mats, count, dtype, P->ds->sms,
                             base + o_umma, umma_bytes, P->d_counters, tune, &g_err);
        if (ust != PE_OK) return ust;
    }
    *out = P.release();
    return PE_OK;
}

// Alg. 4 (FP32 path) after prepare: the steps in blocks of k = restart (the
// last block shorter). Per block: Y = s^2 X X^T (SIMT Gram, split-K for long
// L; s = the normalisation factor in the first block, 1 after), the shift
// Y += shift I in the first block, Q_1 = h_1(Y) = a I + b Y + c Y Y, then for
// each further step P = Y Q, R = Q^T P, H = a I + b R + c R R, Q <- Q H, and
// X <- s Q X (SIMT update kernel with a = 0 and B = Q; the last block stores
// the caller's layout). Q_j of a k-step block is kept in Qb[(k - j) & 1]
// (Qb[0] = DevMat::bfp, Qb[1] = the plan's second Q buffer), so Q_k is in bfp.
int enqueue_fast(Plan* P, cudaStream_t st, int* nk) {
    const PlanKey& k = P->key;
    // one s x s product: its tiles (or K chunks), then the chunks' reduction
    auto product = [&](int list, bool ta, float alpha, float beta, float gamma) -> cudaError_t {
        cudaError_t e = launch_fast_gemm(P->d_fast[list], P->n_fast[list], ta, alpha, beta, gamma, st);
        ++*nk;
        if (e == cudaSuccess && P->n_fred[list]) {
            e = launch_fast_reduce(P->d_fred[list], P->n_fred[list], alpha, beta, gamma, st);
            ++*nk;
        }
        return e;
    };
    int cur = 0;
    for (int t = 0; t < k.T;) {
        const int kb = std::min(k.restart, k.T - t);
        const bool first = (t == 0);
        {
            TraceScope ts(2, st);
            PE_CU(launch_simt_phase(P->d_mats, P->d_tiles[kGram], P->n_tiles[kGram], kGram, 0.f, 0.f, 0.f, cur, 0,
                                    first, P->d_nscale, st));
            ++*nk;
        }
        if (P->n_red) {
            TraceScope ts(9, st);
            PE_CU(launch_simt_gram_reduce(P->d_mats, P->d_red, P->n_red, first, P->d_nscale, st));
            ++*nk;
        }
        if (first && k.shift != 0.f) {
            TraceScope ts(11, st);
            PE_CU(launch_fast_shift(P->d_mats, (int)P->mats.size(), k.shift, st));
            ++*nk;
        }
        {
            TraceScope ts(10, st);   // the block's s x s products
            const float a = k.coef[3 * t], b = k.coef[3 * t + 1], c = k.coef[3 * t + 2];
            PE_CU(product(Plan::kFSq0 + ((kb - 1) & 1), false, c, b, a));
            for (int j = 2; j <= kb; ++j) {
                const int r = 3 * (t + j - 1);
                const float aj = k.coef[r], bj = k.coef[r + 1], cj = k.coef[r + 2];
                const int p = (kb - j + 1) & 1;   // the buffer holding Q_{j-1}
                PE_CU(product(Plan::kFP0 + p, false, 1.f, 0.f, 0.f));
                PE_CU(product(Plan::kFR0 + p, true, 1.f, 0.f, 0.f));
                PE_CU(product(Plan::kFH, false, cj, bj, aj));
                PE_CU(product(Plan::kFQ0 + p, false, 1.f, 0.f, 0.f));
            }
        }
        {
            TraceScope tu(4, st);
            PE_CU(launch_simt_phase(P->d_mats, P->d_tiles[kApply], P->n_tiles[kApply], kApply, 0.f, 0.f, 0.f, cur,
                                    t + kb == k.T, first, P->d_nscale, st));
            ++*nk;
        }
        cur ^= 1;
        t += kb;
    }
    return PE_OK;
}

// Enqueue the whole online stage of a plan on `st`. With `tuning`, only the
// first min(T, 3) steps run and none of them writes the caller's buffer.
int enqueue(Plan* P, cudaStream_t st, bool tuning = false) {
    const PlanKey& k = P->key;
    int nk = 0;
    int outputs = kPrepF32;                                               // FP32
    if (k.dtype == PE_BF16) outputs = kPrepCode;                          // hi + code (compact master)
    if (k.dtype == PE_BF16X3) outputs = kPrepF32 | kPrepBF16 | kPrepBF16Lo;
    if (!k.w.empty()) outputs |= kPrepMuon;                              // fused Muon step: momentum in prepare
    if (tuning) outputs |= kPrepNoMom;                                    // a tuning run leaves M unchanged
    outputs |= kPrepSkipPad;
    {
        TraceScope ts(1, st);
        PE_CU(launch_prepare(P->d_mats, (int)P->mats.size(), P->d_prep, P->n_prep, P->d_partials, k.scale, k.eps, outputs,
                             P->d_nscale, P->ds->status, P->d_counters, P->n_counters, P->d_ticket, st));
    }
    ++nk;
    if (k.restart > 0) {
        const int r = enqueue_fast(P, st, &nk);
        if (r != PE_OK) return r;
        P->kernels_per_run = nk;
        return PE_OK;
    }
    const int T = tuning ? std::min(k.T, 3) : k.T;
    for (int t = 0; t < T; ++t) {
        const float a = k.coef[3 * t], b = k.coef[3 * t + 1], c = k.coef[3 * t + 2];
        const int last = (!tuning && t == k.T - 1);
        if (k.dtype == PE_FP32) {
            for (int ph = 0; ph < 3; ++ph) {
                {
                    TraceScope ts(2 + ph, st);
                    PE_CU(launch_simt_phase(P->d_mats, P->d_tiles[ph], P->n_tiles[ph], ph, a, b, c, t & 1,
                                            last, t == 0, P->d_nscale, st));
                    ++nk;
                }
                if (ph == kGram && P->n_red) {
                    TraceScope ts(9, st);
                    PE_CU(launch_simt_gram_reduce(P->d_mats, P->d_red, P->n_red, t == 0, P->d_nscale, st));
                    ++nk;
                }
            }
        } else {
            const bool phased = (k.flags & PE_BATCH_PHASED) != 0;
            int withhold = (int)g_dbg_withhold;
            int n_launched = 0;
            cudaError_t e = cudaSuccess;
            P->umma.prof = g_dbg_prof;
            if (!phased) {
                TraceScope ts(5, st);
                e = umma_step(&P->umma, t, a, b, c, last, -1, withhold, (uint64_t)g_dbg_wait_ns,
                              P->ds->status, st, &n_launched);
            } else {
                for (int ph = 0; ph < 3 && e == cudaSuccess; ++ph) {
                    TraceScope ts(6 + ph, st);
                    int nl = 0;
                    e = umma_step(&P->umma, t, a, b, c, last, ph, withhold, (uint64_t)g_dbg_wait_ns,
                                  P->ds->status, st, &nl);
                    n_launched += nl;
                }
            }
            if (e != cudaSuccess) return cuda_fail(e, "umma_step");
            nk += n_launched;
        }
    }
    if (tuning) return PE_OK;
    g_dbg_withhold = -1;
    P->kernels_per_run = nk;
    return PE_OK;
}

// ------------------------------------------------------------ autotuner
// The tile schedule of a tcgen05 plan is picked by timing the candidate
// schedules on the plan's own workspace (enqueue with `tuning`: the caller's
// buffer is read by prepare but never written). Results are cached per
// device and shape signature in memory and, when PE_AUTOTUNE_CACHE names a
// file, in that file as JSON lines {"key": "...", "order": n} with
// n = 16 * kernel mode + tile order.

std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const PlanKey& k, const DeviceState* ds) {
    std::string s = "sm" + std::to_string(ds->major) + std::to_string(ds->minor) + "x" + std::to_string(ds->sms) +
                    "|d" + std::to_string(k.dtype) + "|T" + std::to_string(std::min(k.T, 3)) + "|";
    for (int i = 0; i < k.count; ++i) {
        const int64_t m = k.dims[3 * i], n = k.dims[3 * i + 1];
        s += std::to_string(std::min(m, n)) + "x" + std::to_string(std::max(m, n)) + ",";
    }
    if (s.size() > 512) {   // long signatures are hashed
        uint64_t h = 1469598103934665603ull;
        for (unsigned char c : s) h = (h ^ c) * 1099511628211ull;
        s = s.substr(0, 64) + "#" + std::to_string(h);
    }
    return s;
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("PE_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[2048];
    while (fgets(line, sizeof(line), f)) {
        const char* k = strstr(line, "\"key\": \"");
        const char* o = strstr(line, "\"order\": ");
        if (!k || !o) continue;
        k += 8;
        const char* ke = strchr(k, '"');
        if (!ke) continue;
        g_tune[std::string(k, ke - k)] = atoi(o + 9);
    }
    fclose(f);
}

void tune_store(const std::string& key, int order) {
    g_tune[key] = order;
    const char* path = getenv("PE_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"order\": %d}\n", key.c_str(), order);
    fclose(f);
}

int autotune(Plan* P, cudaStream_t st) {
    tune_load();
    const std::string key = tune_key(P->key, P->ds);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
        const int mode = it->second / 16, order = it->second % 16;
        if ((mode != 0 && mode != 2 && mode != 3) || (mode == 2 && P->umma.max_clusters2 < 1) ||
            (mode == 3 && P->umma.max_clusters3 < 1))
            return PE_OK;   // cached on another configuration
        P->umma.mode = mode;
        return umma_schedule(&P->umma, order, &g_err);
    }
    cudaEvent_t a = nullptr, b = nullptr;
    PE_CU(cudaEventCreate(&a));
    PE_CU(cudaEventCreate(&b));
    PE_CU(cudaStreamSynchronize(st));
    int best_order = P->umma.order, best_mode = P->umma.mode;
    int r = PE_OK;
    const int n_orders = (P->key.count >= 8) ? 5 : 2;   // lagged interleaves need several matrices
    std::vector<int> modes;
    if (g_dbg_mode >= 0) modes.push_back(P->umma.mode);
    else {
        modes.push_back(0);
        if (P->umma.max_clusters2 > 0) modes.push_back(2);
        if (P->umma.max_clusters3 > 0) modes.push_back(3);
    }
    // Round robin over the candidates (a warm-up pass, then two timed passes,
    // the faster run of each candidate counts), so that a drift of clocks or
    // power during tuning does not favour the candidates timed first.
    const int ncand = n_orders * (int)modes.size();
    std::vector<float> cand_ms(ncand, 1e30f);
    for (int pass = 0; pass < 3 && r == PE_OK; ++pass) {
        for (int cand = 0; cand < ncand && r == PE_OK; ++cand) {
            P->umma.mode = modes[cand / n_orders];
            r = umma_schedule(&P->umma, cand % n_orders, &g_err);
            if (r != PE_OK) break;
            cudaEventRecord(a, st);
            r = enqueue(P, st, true);
            cudaEventRecord(b, st);
            if (cudaEventSynchronize(b) != cudaSuccess) r = cuda_fail(cudaGetLastError(), "autotune");
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            if (pass > 0 && t < cand_ms[cand]) cand_ms[cand] = t;
        }
    }
    if (r == PE_OK) {
        int bc = 0;
        for (int cand = 1; cand < ncand; ++cand)
            if (cand_ms[cand] < cand_ms[bc]) bc = cand;
        best_mode = modes[bc / n_orders];
        best_order = bc % n_orders;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r != PE_OK) return r;
    tune_store(key, 16 * best_mode + best_order);
    P->umma.mode = best_mode;
    return umma_schedule(&P->umma, best_order, &g_err);
}

int get_plan(const PlanKey& key, cudaStream_t st, Plan** out, bool* fresh) {
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
        if ((*it)->key == key) {
            g_plans.splice(g_plans.begin(), g_plans, it);
            *out = g_plans.front().get();
            *fresh = false;
            return PE_OK;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    PE_CU(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(PE_EINVAL, "no cached plan for this call while the stream is capturing; "
                               "run the call once before capturing it");
    Plan* p = nullptr;
    int r = build_plan(key, &p);
    if (r != PE_OK) return r;
    g_plans.emplace_front(p);
    while (g_plans.size() > kMaxPlans) {
        cudaDeviceSynchronize();
        g_plans.pop_back();
    }
    *out = p;
    *fresh = true;
    return PE_OK;
}

int run(void* const* X, const int64_t* m, const int64_t* n, const int64_t* ld, int count, int io,
        const double* table, int T, int dtype, double scale, double eps, unsigned flags, void* stream,
        void* const* Mom = nullptr, void* const* W = nullptr, double beta = 0.0, double lr = 0.0,
        int restart = 0, double shift = 0.0) {
    if (!X || !m || !n) return fail(PE_EINVAL, "NULL argument");
    if (count < 1 || count > kMaxMatrices) return fail(PE_EINVAL, "count must be in 1..4096");
    if (!table) return fail(PE_EINVAL, "table is NULL");
    if (T < 1 || T > kMaxSteps) return fail(PE_EINVAL, "T must be in 1..64");
    if (dtype != PE_FP32 && dtype != PE_BF16 && dtype != PE_BF16X3) return fail(PE_EINVAL, "bad dtype");
    if (io != PE_IO_FP32 && io != PE_IO_BF16) return fail(PE_EINVAL, "bad io_type");
    if (!(std::isfinite(scale) && scale > 0) || !(std::isfinite(eps) && eps >= 0))
        return fail(PE_EINVAL, "norm_scale must be > 0 and norm_eps >= 0");
    PlanKey key;
    key.dtype = dtype;
    key.T = T;
    key.io = io;
    key.count = count;
    key.flags = flags;
    key.scale = (float)scale;
    key.eps = (float)eps;
    key.ptrs.resize(count);
    key.dims.resize(3 * count);
    for (int i = 0; i < count; ++i) {
        if (!X[i]) return fail(PE_EINVAL, "matrix pointer " + std::to_string(i) + " is NULL");
        const int64_t ldi = ld ? ld[i] : n[i];
        if (m[i] < 1 || n[i] < 1) return fail(PE_EINVAL, "sizes must be >= 1");
        if (m[i] > (1 << 20) || n[i] > (1 << 20) || m[i] * n[i] > (int64_t)1 << 31)
            return fail(PE_EINVAL, "matrix too large (m, n <= 2^20, m*n <= 2^31)");
        if (ldi < n[i]) return fail(PE_EINVAL, "ld must be >= n");
        const size_t esz = io == PE_IO_BF16 ? 2 : 4;
        if (reinterpret_cast<uintptr_t>(X[i]) % esz) return fail(PE_EINVAL, "misaligned matrix pointer");
        key.ptrs[i] = reinterpret_cast<uintptr_t>(X[i]);
        key.dims[3 * i] = m[i];
        key.dims[3 * i + 1] = n[i];
        key.dims[3 * i + 2] = ldi;
    }
    key.coef.resize(3 * T);
    for (int i = 0; i < 3 * T; ++i) {
        if (!std::isfinite(table[i])) return fail(PE_EINVAL, "non-finite coefficient in table");
        key.coef[i] = (float)table[i];
    }
    if (restart) {
        if (restart < 1 || restart > kMaxSteps) return fail(PE_EINVAL, "restart must be in 1..64");
        if (!(std::isfinite(shift) && shift >= 0)) return fail(PE_EINVAL, "shift must be finite and >= 0");
        if (dtype != PE_FP32) return fail(PE_EUNSUPPORTED, "the fast rectangular iteration runs on PE_FP32");
        key.restart = restart;
        key.shift = (float)shift;
    }
    if (W) {
        if (!Mom) return fail(PE_EINVAL, "momentum pointer array is NULL");
        if (io != PE_IO_FP32) return fail(PE_EINVAL, "the fused Muon step takes FP32 matrices");
        if (!(std::isfinite(beta) && beta >= 0 && beta <= 1)) return fail(PE_EINVAL, "beta must be in [0, 1]");
        if (!std::isfinite(lr)) return fail(PE_EINVAL, "lr must be finite");
        key.mom.resize(count);
        key.w.resize(count);
        for (int i = 0; i < count; ++i) {
            if (!Mom[i] || !W[i]) return fail(PE_EINVAL, "momentum or weight pointer " + std::to_string(i) + " is NULL");
            if (reinterpret_cast<uintptr_t>(Mom[i]) % 4 || reinterpret_cast<uintptr_t>(W[i]) % 4)
                return fail(PE_EINVAL, "misaligned momentum or weight pointer");
            key.mom[i] = reinterpret_cast<uintptr_t>(Mom[i]);
            key.w[i] = reinterpret_cast<uintptr_t>(W[i]);
        }
        key.beta = (float)beta;
        key.lr = (float)lr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    PE_CU(cudaGetDevice(&key.dev));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Plan* P = nullptr;
    bool fresh = false;
    int r = get_plan(key, st, &P, &fresh);
    if (r != PE_OK) return r;
    if (fresh && dtype != PE_FP32 && !(flags & PE_BATCH_NO_TUNE) && g_dbg_order < 0) {
        r = autotune(P, st);
        if (r != PE_OK) return r;
    }
    const bool use_graph = !(flags & PE_BATCH_NO_GRAPH) && count > 1;
    if (!use_graph || g_dbg_withhold >= 0 || g_trace || g_dbg_prof) {
        r = enqueue(P, st);
        if (r != PE_OK) return r;
        g_launches += P->kernels_per_run;
        return PE_OK;
    }
    if (!P->exec) {
        cudaGraph_t g = nullptr;
        cudaStream_t cap = P->ds->cap;
        PE_CU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        r = enqueue(P, cap);
        cudaError_t ee = cudaStreamEndCapture(cap, &g);
        if (r != PE_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
        ee = cudaGraphInstantiate(&P->exec, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) {
            P->exec = nullptr;
            return cuda_fail(ee, "cudaGraphInstantiate");
        }
    }
    PE_CU(cudaGraphLaunch(P->exec, st));
    g_launches += P->kernels_per_run;
    return PE_OK;
}

// ---------------------------------------------------- host-buffer entry
// pe_polar_batched_host: device staging buffers per shape set, and the copies
// pipelined with the grouped compute: group g's host->device copies run on
// one copy stream, its compute on the caller's stream once they land, and its
// device->host copies on a second copy stream, so the link works in both
// directions while the tensor cores work on another group.

struct HostPlan {
    int dev = 0;
    std::vector<int64_t> dims;       // m, n per matrix
    std::vector<size_t> off;         // byte offset of matrix i in mem
    char* mem = nullptr;
    cudaStream_t c_in = nullptr, c_out = nullptr;
    std::vector<cudaEvent_t> ev;     // start, done, and 2 per group
    ~HostPlan() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (c_in) cudaStreamDestroy(c_in);
        if (c_out) cudaStreamDestroy(c_out);
        if (mem) cudaFree(mem);
    }
};
std::list<std::unique_ptr<HostPlan>> g_hplans;
constexpr size_t kMaxHostPlans = 4;

int host_plan(const std::vector<int64_t>& dims, int ngroups, HostPlan** out) {
    int dev = 0;
    PE_CU(cudaGetDevice(&dev));
    for (auto it = g_hplans.begin(); it != g_hplans.end(); ++it) {
        if ((*it)->dev == dev && (*it)->dims == dims && (int)(*it)->ev.size() >= 2 + 2 * ngroups) {
            g_hplans.splice(g_hplans.begin(), g_hplans, it);
            *out = g_hplans.front().get();
            return PE_OK;
        }
    }
    auto H = std::make_unique<HostPlan>();
    H->dev = dev;
    H->dims = dims;
    size_t tot = 0;
    for (size_t i = 0; i < dims.size() / 2; ++i) {
        H->off.push_back(tot);
        tot += round_up((size_t)(dims[2 * i] * dims[2 * i + 1]) * sizeof(float), 256);
    }
    if (g_dbg_fail_alloc) {
        g_dbg_fail_alloc = false;
        return fail(PE_ENOMEM, "staging allocation failed (injected)");
    }
    cudaError_t e = cudaMalloc(&H->mem, tot);
    if (e != cudaSuccess) {
        cudaGetLastError();
        H->mem = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? PE_ENOMEM : PE_ECUDA,
                    std::string("staging allocation of ") + std::to_string(tot) + " bytes failed");
    }
    PE_CU(cudaStreamCreateWithFlags(&H->c_in, cudaStreamNonBlocking));
    PE_CU(cudaStreamCreateWithFlags(&H->c_out, cudaStreamNonBlocking));
    H->ev.assign(2 + 2 * std::max(ngroups, 4), nullptr);
    for (cudaEvent_t& ev : H->ev) PE_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    g_hplans.emplace_front(std::move(H));
    while (g_hplans.size() > kMaxHostPlans) {
        cudaDeviceSynchronize();
        g_hplans.pop_back();
    }
    *out = g_hplans.front().get();
    return PE_OK;
}

int run_host(const void* const* Hin, void* const* Hout, const int64_t* m, const int64_t* n, int count,
             const double* table, int T, int dtype, int ngroups, void* stream) {
    if (!Hin || !Hout || !m || !n) return fail(PE_EINVAL, "NULL argument");
    if (count < 1 || count > kMaxMatrices) return fail(PE_EINVAL, "count must be in 1..4096");
    if (ngroups < 0) return fail(PE_EINVAL, "ngroups must be >= 0");
    std::vector<int64_t> dims(2 * count);
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (!Hin[i] || !Hout[i]) return fail(PE_EINVAL, "host pointer " + std::to_string(i) + " is NULL");
        if (m[i] < 1 || n[i] < 1) return fail(PE_EINVAL, "sizes must be >= 1");
        if (m[i] > (1 << 20) || n[i] > (1 << 20) || m[i] * n[i] > (int64_t)1 << 31)
            return fail(PE_EINVAL, "matrix too large (m, n <= 2^20, m*n <= 2^31)");
        dims[2 * i] = m[i];
        dims[2 * i + 1] = n[i];
        total += (size_t)(m[i] * n[i]);
    }
    const int ng = std::min(count, ngroups > 0 ? ngroups : 6);
    // contiguous groups balanced by bytes
    std::vector<int> cut(ng + 1, count);
    cut[0] = 0;
    {
        size_t acc = 0;
        int g = 1;
        for (int i = 0; i < count && g < ng; ++i) {
            acc += (size_t)(m[i] * n[i]);
            if (acc * ng >= total * g && i + 1 < count) cut[g++] = i + 1;
        }
        for (; g < ng; ++g) cut[g] = count;   // fewer usable cuts than groups: empty groups
    }
    HostPlan* H = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        int r = host_plan(dims, ng, &H);
        if (r != PE_OK) return r;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PE_CU(cudaEventRecord(H->ev[0], st));
    PE_CU(cudaStreamWaitEvent(H->c_in, H->ev[0], 0));
    PE_CU(cudaStreamWaitEvent(H->c_out, H->ev[0], 0));
    std::vector<void*> dptr(count);
    for (int i = 0; i < count; ++i) dptr[i] = H->mem + H->off[i];
    for (int g = 0; g < ng; ++g) {
        const int a = cut[g], b = cut[g + 1];
        if (a >= b) continue;
        for (int i = a; i < b; ++i)
            PE_CU(cudaMemcpyAsync(dptr[i], Hin[i], (size_t)(m[i] * n[i]) * sizeof(float), cudaMemcpyHostToDevice,
                                  H->c_in));
        PE_CU(cudaEventRecord(H->ev[2 + 2 * g], H->c_in));
        PE_CU(cudaStreamWaitEvent(st, H->ev[2 + 2 * g], 0));
        int r = run(dptr.data() + a, m + a, n + a, nullptr, b - a, PE_IO_FP32, table, T, dtype, 1.01, 1e-7, 0,
                    stream);
        if (r != PE_OK) return r;
        PE_CU(cudaEventRecord(H->ev[3 + 2 * g], st));
        PE_CU(cudaStreamWaitEvent(H->c_out, H->ev[3 + 2 * g], 0));
        for (int i = a; i < b; ++i)
            PE_CU(cudaMemcpyAsync(Hout[i], dptr[i], (size_t)(m[i] * n[i]) * sizeof(float), cudaMemcpyDeviceToHost,
                                  H->c_out));
    }
    PE_CU(cudaEventRecord(H->ev[1], H->c_out));
    PE_CU(cudaStreamWaitEvent(st, H->ev[1], 0));
    return PE_OK;
}

// ------------------------------------------------------ long-side split
// One rank's block of a matrix split along its long side (pe_split_*): a
// dedicated single-matrix plan (orientation fixed by the caller, phased
// launches, no graph, no tuning), stepped by the host one phase at a time so
// that the caller can sum the partial norms and Grams across ranks.

struct Split {
    std::unique_ptr<Plan> plan;
    cudaStream_t st = nullptr;
    int s = 0;             // shared short side
    float s0 = 0.f;        // normalisation factor from the global norm
    bool norm_set = false;
    int next_gram = 0, next_step = 0;
    std::vector<double> partials;
};

int split_open(void* X, int64_t rows, int64_t cols, int short_is_rows, const double* table, int T, int dtype,
               void* stream, Split** out) {
    if (!out) return fail(PE_EINVAL, "handle pointer is NULL");
    *out = nullptr;
    if (!X || !table) return fail(PE_EINVAL, "NULL argument");
    if (dtype == PE_BF16X3) return fail(PE_EUNSUPPORTED, "the long-side split supports PE_FP32 and PE_BF16");
    if (dtype != PE_FP32 && dtype != PE_BF16) return fail(PE_EINVAL, "bad dtype");
    if (T < 1 || T > kMaxSteps) return fail(PE_EINVAL, "T must be in 1..64");
    if (rows < 1 || cols < 1) return fail(PE_EINVAL, "sizes must be >= 1");
    if (rows > (1 << 20) || cols > (1 << 20) || rows * cols > (int64_t)1 << 31)
        return fail(PE_EINVAL, "matrix too large (rows, cols <= 2^20, rows*cols <= 2^31)");
    if (reinterpret_cast<uintptr_t>(X) % 4) return fail(PE_EINVAL, "misaligned matrix pointer");
    PlanKey key;
    key.dtype = dtype;
    key.T = T;
    key.io = PE_IO_FP32;
    key.count = 1;
    key.flags = kFlagSplit | (short_is_rows ? 0u : kFlagSplitShortCols) | PE_BATCH_NO_GRAPH | PE_BATCH_PHASED |
                PE_BATCH_NO_TUNE;
    key.scale = 1.01f;
    key.eps = 1e-7f;
    key.ptrs = {reinterpret_cast<uintptr_t>(X)};
    key.dims = {rows, cols, cols};
    key.coef.resize(3 * T);
    for (int i = 0; i < 3 * T; ++i) {
        if (!std::isfinite(table[i])) return fail(PE_EINVAL, "non-finite coefficient in table");
        key.coef[i] = (float)table[i];
    }
    PE_CU(cudaGetDevice(&key.dev));
    Plan* p = nullptr;
    int r = build_plan(key, &p);
    if (r != PE_OK) return r;
    auto S = std::make_unique<Split>();
    S->plan.reset(p);
    S->st = reinterpret_cast<cudaStream_t>(stream);
    S->s = p->mats[0].s;
    *out = S.release();
    return PE_OK;
}

int split_sumsq(Split* S, double* sumsq) {
    if (!S || !sumsq) return fail(PE_EINVAL, "NULL argument");
    Plan* P = S->plan.get();
    const PlanKey& k = P->key;
    const int outputs = ((k.dtype == PE_BF16) ? kPrepCode : kPrepF32) | kPrepSkipPad;
    PE_CU(launch_prepare(P->d_mats, 1, P->d_prep, P->n_prep, P->d_partials, k.scale, k.eps, outputs,
                         P->d_nscale, P->ds->status, P->d_counters, P->n_counters, P->d_ticket, S->st));
    S->partials.resize(P->n_prep);
    PE_CU(cudaMemcpyAsync(S->partials.data(), P->d_partials, sizeof(double) * P->n_prep, cudaMemcpyDeviceToHost,
                          S->st));
    PE_CU(cudaStreamSynchronize(S->st));
    // the order of the single-device normalisation: 32 strided lane sums,
    // then the butterfly that leaves lane 0 with the total
    double lanes[32];
    for (int l = 0; l < 32; ++l) {
        lanes[l] = 0.0;
        for (size_t i = l; i < S->partials.size(); i += 32) lanes[l] += S->partials[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        double nxt[32];
        for (int l = 0; l < 32; ++l) nxt[l] = lanes[l] + lanes[l ^ o];
        for (int l = 0; l < 32; ++l) lanes[l] = nxt[l];
    }
    *sumsq = lanes[0];
    S->norm_set = false;
    S->next_gram = S->next_step = 0;
    return PE_OK;
}

int split_set_norm(Split* S, double total) {
    if (!S) return fail(PE_EINVAL, "NULL handle");
    if (!(std::isfinite(total) && total >= 0)) return fail(PE_EINVAL, "total_sumsq must be finite and >= 0");
    Plan* P = S->plan.get();
    S->s0 = (float)(1.0 / ((double)P->key.scale * std::sqrt(total) + (double)P->key.eps));
    PE_CU(cudaMemcpyAsync(P->d_nscale, &S->s0, sizeof(float), cudaMemcpyHostToDevice, S->st));
    S->norm_set = true;
    return PE_OK;
}

int split_gram(Split* S, int t, float* A, int64_t lda) {
    if (!S || !A) return fail(PE_EINVAL, "NULL argument");
    Plan* P = S->plan.get();
    const PlanKey& k = P->key;
    if (!S->norm_set) return fail(PE_EINVAL, "pe_split_set_norm must come before the first Gram");
    if (t != S->next_gram || t != S->next_step || t >= k.T)
        return fail(PE_EINVAL, "steps must run in order: gram(t) then step(t), t = 0 .. T-1");
    if (lda < S->s) return fail(PE_EINVAL, "lda must be >= s");
    const DevMat& M = P->mats[0];
    const float a = k.coef[3 * t], b = k.coef[3 * t + 1], c = k.coef[3 * t + 2];
    if (k.dtype == PE_FP32) {
        PE_CU(launch_simt_phase(P->d_mats, P->d_tiles[kGram], P->n_tiles[kGram], kGram, a, b, c, t & 1, 0, t == 0,
                                P->d_nscale, S->st));
    } else {
        int nl = 0;
        cudaError_t e = umma_step(&P->umma, t, a, b, c, 0, kGram, -1, (uint64_t)g_dbg_wait_ns, P->ds->status,
                                  S->st, &nl);
        if (e != cudaSuccess) return cuda_fail(e, "umma_step (split Gram)");
    }
    PE_CU(cudaMemcpy2DAsync(A, sizeof(float) * lda, M.af, sizeof(float) * M.sp, sizeof(float) * S->s, S->s,
                            cudaMemcpyDeviceToDevice, S->st));
    S->next_gram = t + 1;
    return PE_OK;
}

int split_step(Split* S, int t, const float* A, int64_t lda) {
    if (!S || !A) return fail(PE_EINVAL, "NULL argument");
    Plan* P = S->plan.get();
    const PlanKey& k = P->key;
    if (t != S->next_step || S->next_gram != t + 1) return fail(PE_EINVAL, "pe_split_gram(t) must come before pe_split_step(t)");
    if (lda < S->s) return fail(PE_EINVAL, "lda must be >= s");
    const DevMat& M = P->mats[0];
    const float a = k.coef[3 * t], b = k.coef[3 * t + 1], c = k.coef[3 * t + 2];
    const int last = (t == k.T - 1);
    if (k.dtype == PE_FP32) {
        PE_CU(cudaMemcpy2DAsync(M.af, sizeof(float) * M.sp, A, sizeof(float) * lda, sizeof(float) * S->s, S->s,
                                cudaMemcpyDeviceToDevice, S->st));
        for (int ph = kSquare; ph <= kApply; ++ph)
            PE_CU(launch_simt_phase(P->d_mats, P->d_tiles[ph], P->n_tiles[ph], ph, a, b, c, t & 1, last, t == 0,
                                    P->d_nscale, S->st));
    } else {
        PE_CU(launch_split_load_a(A, lda, S->s, M.sp, M.ah, S->st));
        PE_CU(launch_split_d(A, lda, S->s, M.sp, M.btr, S->st));
        for (int ph = kSquare; ph <= kApply; ++ph) {
            int nl = 0;
            cudaError_t e = umma_step(&P->umma, t, a, b, c, last, ph, -1, (uint64_t)g_dbg_wait_ns, P->ds->status,
                                      S->st, &nl);
            if (e != cudaSuccess) return cuda_fail(e, "umma_step (split step)");
        }
    }
    S->next_step = t + 1;
    return PE_OK;
}

}  // namespace

void set_last_error(const char* msg) { g_err = msg; }

}  // namespace pe

struct pe_split_s {
    pe::Split* impl;
};

extern "C" {

int pe_version(void) { return 10000; }

int pe_coeffs(int degree, double l, int T, double safety, double* coeffs, double* bounds) {
    return pe_coeffs_ex(degree, l, T, safety, -1.0, 0u, coeffs, bounds, nullptr);
}

int pe_coeffs_ex(int degree, double l, int T, double safety, double cushion, unsigned flags,
                 double* coeffs, double* bounds, int* remez_iters) {
    const char* why = "";
    int r = pe::coeffs_table(degree, l, T, safety, cushion, flags, coeffs, bounds, remez_iters, &why);
    if (r != PE_OK) pe::g_err = why;
    return r;
}

int pe_polar(void* X, int64_t m, int64_t n, const double* table, int T, int dtype, void* stream) {
    return pe_polar_ex(X, m, n, n, PE_IO_FP32, table, T, dtype, 1.01, 1e-7, stream);
}

int pe_polar_ex(void* X, int64_t m, int64_t n, int64_t ld, int io_type, const double* table, int T,
                int dtype, double norm_scale, double norm_eps, void* stream) {
    void* xs[1] = {X};
    int64_t ms[1] = {m}, ns[1] = {n}, lds[1] = {ld};
    return pe::run(xs, ms, ns, lds, 1, io_type, table, T, dtype, norm_scale, norm_eps,
                   PE_BATCH_NO_GRAPH, stream);
}

int pe_polar_batched(void* const* X, const int64_t* m, const int64_t* n, int count,
                     const double* table, int T, int dtype, void* stream) {
    return pe::run(X, m, n, nullptr, count, PE_IO_FP32, table, T, dtype, 1.01, 1e-7, 0u, stream);
}

int pe_polar_batched_ex(void* const* X, const int64_t* m, const int64_t* n, int count, int io_type,
                        const double* table, int T, int dtype, double norm_scale, double norm_eps,
                        unsigned flags, void* stream) {
    return pe::run(X, m, n, nullptr, count, io_type, table, T, dtype, norm_scale, norm_eps, flags,
                   stream);
}

int pe_polar_fast_batched(void* const* X, const int64_t* m, const int64_t* n, int count, const double* table, int T,
                          int restart, double shift, double norm_eps, int dtype, unsigned flags, void* stream) {
    if (restart < 1) return pe::fail(PE_EINVAL, "restart must be in 1..64");
    return pe::run(X, m, n, nullptr, count, PE_IO_FP32, table, T, dtype, 1.01, norm_eps, flags, stream, nullptr,
                   nullptr, 0.0, 0.0, restart, shift);
}

int pe_polar_fast(void* X, int64_t m, int64_t n, const double* table, int T, int restart, int dtype, void* stream) {
    void* xs[1] = {X};
    int64_t ms[1] = {m}, ns[1] = {n};
    return pe_polar_fast_batched(xs, ms, ns, 1, table, T, restart, 1e-3, 1e-3, dtype, PE_BATCH_NO_GRAPH, stream);
}

int pe_polar_batched_host(const void* const* Hin, void* const* Hout, const int64_t* m, const int64_t* n, int count,
                          const double* table, int T, int dtype, int ngroups, void* stream) {
    return pe::run_host(Hin, Hout, m, n, count, table, T, dtype, ngroups, stream);
}

int pe_sync_status(void* stream) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    pe::DeviceState* d = nullptr;
    int r = pe::device_state(&d);
    if (r != PE_OK) return r;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pe::cuda_fail(e, "cudaStreamSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, d->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pe::cuda_fail(e, "reading the status word");
    e = cudaMemset(d->status, 0, sizeof(int));
    if (e != cudaSuccess) return pe::cuda_fail(e, "clearing the status word");
    if (h & 1) return pe::fail(PE_ETIMEOUT, "a bounded device wait expired; results are invalid");
    if (h & 4) return pe::fail(PE_ETIMEOUT, "a pipeline wait of a tcgen05 kernel expired; results are invalid");
    if (h & 8) return pe::fail(PE_ECUDA, "the CTAs of a 2-SM pair got different TMEM bases; results are invalid");
    if (h & 2) return pe::fail(PE_ECUDA, "non-finite Frobenius norm in the input");
    return PE_OK;
}

int64_t pe_launch_count(void) { return pe::g_launches.load(); }

int pe_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    for (auto& r : pe::g_trace_recs) {
        cudaEventSynchronize(r.b);
        pe::g_event_pool.push_back(r.a);
        pe::g_event_pool.push_back(r.b);
    }
    pe::g_trace_recs.clear();
    pe::g_trace = on != 0;
    return PE_OK;
}

int pe_trace_read(int64_t* launches, double* ms, int nkinds) {
    if (!launches || !ms || nkinds < 1) return pe::fail(PE_EINVAL, "bad trace_read arguments");
    std::lock_guard<std::mutex> lk(pe::g_mu);
    for (int k = 0; k < nkinds; ++k) { launches[k] = 0; ms[k] = 0.0; }
    for (auto& r : pe::g_trace_recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return pe::cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return pe::cuda_fail(e, "cudaEventElapsedTime");
        if (r.kind < nkinds) {
            launches[r.kind] += 1;
            ms[r.kind] += t;
        }
    }
    return PE_OK;
}

const char* pe_last_error(void) { return pe::g_err.c_str(); }

void pe_release(void) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    if (!pe::g_plans.empty() || !pe::g_hplans.empty()) cudaDeviceSynchronize();
    pe::g_plans.clear();
    pe::g_hplans.clear();
}

int pe_split_open(void* X, int64_t rows, int64_t cols, int short_is_rows, const double* table, int T, int dtype,
                  void* stream, pe_split_t* handle) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    if (!handle) return pe::fail(PE_EINVAL, "handle pointer is NULL");
    *handle = nullptr;
    pe::Split* S = nullptr;
    int r = pe::split_open(X, rows, cols, short_is_rows, table, T, dtype, stream, &S);
    if (r != PE_OK) return r;
    *handle = new pe_split_s{S};
    return PE_OK;
}

int pe_split_sumsq(pe_split_t h, double* sumsq) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    return pe::split_sumsq(h ? h->impl : nullptr, sumsq);
}

int pe_split_set_norm(pe_split_t h, double total_sumsq) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    return pe::split_set_norm(h ? h->impl : nullptr, total_sumsq);
}

int pe_split_gram(pe_split_t h, int t, float* A, int64_t lda) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    return pe::split_gram(h ? h->impl : nullptr, t, A, lda);
}

int pe_split_step(pe_split_t h, int t, const float* A, int64_t lda) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    return pe::split_step(h ? h->impl : nullptr, t, A, lda);
}

int pe_split_close(pe_split_t h) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    if (!h) return pe::fail(PE_EINVAL, "NULL handle");
    cudaError_t e = cudaStreamSynchronize(h->impl->st);
    delete h->impl;
    delete h;
    if (e != cudaSuccess) return pe::cuda_fail(e, "cudaStreamSynchronize");
    return PE_OK;
}

int pe_muon_batched(void* const* W, void* const* G, void* const* M, const int64_t* m, const int64_t* n, int count,
                    double beta, double lr, const double* table, int T, int dtype, unsigned flags, void* stream) {
    if (!W || !G || !M) return pe::fail(PE_EINVAL, "NULL pointer array");
    return pe::run(G, m, n, nullptr, count, PE_IO_FP32, table, T, dtype, 1.01, 1e-7, flags, stream, M, W, beta, lr);
}

int pe_debug_set(int key, int64_t value) {
    std::lock_guard<std::mutex> lk(pe::g_mu);
    switch (key) {
        case 1: pe::g_dbg_withhold = value; return PE_OK;
        case 2: pe::g_dbg_wait_ns = value < 0 ? 0 : value; return PE_OK;
        case 3: pe::g_dbg_fail_alloc = value != 0; return PE_OK;
        case 4: pe::g_dbg_prof = reinterpret_cast<void*>(value); return PE_OK;
        case 5: pe::g_dbg_bk = (int)value; return PE_OK;
        case 6: pe::g_dbg_order = (int)value; return PE_OK;
        case 7:
            if (value != -1 && value != 0 && value != 2 && value != 3)
                return pe::fail(PE_EINVAL, "kernel mode must be -1, 0, 2 or 3");
            pe::g_dbg_mode = (int)value;
            return PE_OK;
        case 8: pe::g_dbg_nacc = (int)value; return PE_OK;
        case 9: pe::g_dbg_nopair = value != 0; return PE_OK;
        default: return pe::fail(PE_EINVAL, "unknown debug key");
    }
}

}  // extern "C"
