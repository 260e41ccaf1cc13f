// Spectrum-aware initialisation for matrices with one dominant singular
// value (App. H, the case k = 1):
//   1. X_0 = G / (1.01 ||G||_F + 1e-7) on the short side (s x L), f = ||X_0||_F;
//   2. a lower bound z <= sigma_1(X_0) by the power method (subspace
//      iteration with one vector) on the s x s matrix X_0 X_0^T from a
//      caller-given start v0: v <- X_0 X_0^T v / ||.||, z = ||X_0^T v||;
//   3. the Frobenius identity gives sigma_1 in [z, f] and every other
//      singular value <= w = sqrt(f^2 - z^2); when the intervals are disjoint
//      the odd cubic p(x) = a x + b x^3 with p(w) = p(z) = 1 (Eq. init_poly,
//      written for f = 1; here that polynomial of x / f) maps the spectrum
//      into [min(l / w, p(f)), 1], and Polar Express continues from there;
//      otherwise T + 1 ordinary steps. Two options that the appendix does not
//      have: a relative shrink of z before use (pe_polar_spectrum_aware
//      shrinks its FP32 bound by 1e-5 so that rounding cannot lift it above
//      sigma_1), and a gate that keeps the cubic only when the composition
//      after it reaches a better final greedy bound than the plain one with
//      one more step.
// The power method is memory-bound matrix-vector work on G itself (two
// passes per iteration); its kernels are plain coalesced FP32 streams with
// deterministic reductions (fixed summation order, FP64 norms).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pe_internal.h"

namespace pe {
namespace {

constexpr int kRowWarps = 8;        // rows per block of the row-dot kernel (one warp each)
constexpr int kColThreads = 256;    // columns-per-block / 4 (vector) of the column kernel
constexpr int kColRows = 64;        // rows per block of the column kernel
constexpr double kZSafetyFp32 = 1e-5;   // relative shrink of an FP32 bound z before use

// out[i] = sum_j M[i, j] x[j] for the m rows of M (m x n row-major); one warp per row
__global__ void rowdot_kernel(const float* __restrict__ M, int64_t m, int64_t n, const float* __restrict__ x,
                              float* __restrict__ out, int vec) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
    if (i >= m) return;
    const float* row = M + i * n;
    float acc = 0.f;
    if (vec) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
        const float4* x4 = reinterpret_cast<const float4*>(x);
        for (int64_t j = lane; j < n / 4; j += 32) {
            const float4 a = __ldcs(r4 + j), b = x4[j];
            acc = fmaf(a.x, b.x, acc);
            acc = fmaf(a.y, b.y, acc);
            acc = fmaf(a.z, b.z, acc);
            acc = fmaf(a.w, b.w, acc);
        }
    } else {
        for (int64_t j = lane; j < n; j += 32) acc = fmaf(__ldcs(row + j), x[j], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = acc;
}

// part[rb * n + j] = sum over the rows of block rb of M[i, j] x[i]
__global__ void coldot_partial_kernel(const float* __restrict__ M, int64_t m, int64_t n,
                                      const float* __restrict__ x, float* __restrict__ part, int vec) {
    const int64_t rb = blockIdx.y;
    const int64_t r0 = rb * kColRows, r1 = std::min<int64_t>(m, r0 + kColRows);
    if (vec) {
        const int64_t j4 = (int64_t)blockIdx.x * kColThreads + threadIdx.x;   // float4 column group
        if (j4 >= n / 4) return;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = r0; i < r1; ++i) {
            const float4 a = __ldcs(reinterpret_cast<const float4*>(M + i * n) + j4);
            const float xi = x[i];
            acc.x = fmaf(a.x, xi, acc.x);
            acc.y = fmaf(a.y, xi, acc.y);
            acc.z = fmaf(a.z, xi, acc.z);
            acc.w = fmaf(a.w, xi, acc.w);
        }
        reinterpret_cast<float4*>(part + rb * n)[j4] = acc;
    } else {
        const int64_t j = (int64_t)blockIdx.x * kColThreads + threadIdx.x;
        if (j >= n) return;
        float acc = 0.f;
        for (int64_t i = r0; i < r1; ++i) acc = fmaf(__ldcs(M + i * n + j), x[i], acc);
        part[rb * n + j] = acc;
    }
}

// out[j] = sum_rb part[rb * n + j], in block order
__global__ void coldot_reduce_kernel(const float* __restrict__ part, int64_t nrb, int64_t n, float* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float acc = 0.f;
    for (int64_t rb = 0; rb < nrb; ++rb) acc += part[rb * n + j];
    out[j] = acc;
}

// *res = sum_i v[i]^2 in FP64 (one block of 1024 threads, fixed order)
__global__ void sumsq_kernel(const float* __restrict__ v, int64_t len, double* __restrict__ res) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const double t = (double)v[i];
        acc += t * t;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *res = red[0];
}

// per-block FP64 partial sums of M's squares (FP32 within a thread's 4-element groups)
__global__ void frob_partial_kernel(const float* __restrict__ M, int64_t total, double* __restrict__ part, int vec) {
    __shared__ double red[256];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const float4* M4 = reinterpret_cast<const float4*>(M);
        for (int64_t k = t0; k < total / 4; k += stride) {
            const float4 a = __ldcs(M4 + k);
            acc += (double)(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
        }
    } else {
        for (int64_t k = t0; k < total; k += stride) {
            const float a = __ldcs(M + k);
            acc += (double)(a * a);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* __restrict__ res) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += part[k];
        *res = acc;
    }
}

// v *= 1 / sqrt(*nrm2) (v unchanged when the norm is zero)
__global__ void scale_kernel(float* __restrict__ v, int64_t len, const double* __restrict__ nrm2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double q = *nrm2;
    if (i >= len || !(q > 0.0)) return;
    v[i] = (float)((double)v[i] / sqrt(q));
}

int sfail(int code, const std::string& msg) {
    set_last_error(msg.c_str());
    return code;
}

int scuda(cudaError_t e, const char* what) {
    set_last_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return PE_ECUDA;
}

#define PE_SCU(call)                                       \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return scuda(_e, #call);    \
    } while (0)

// device buffers of one bound computation, freed on every exit path
struct Bufs {
    float *v = nullptr, *y = nullptr, *part = nullptr;
    double* d = nullptr;   // [0] ||G||^2, [1] ||v||^2 scratch, [2] ||y||^2 final, then frob partials
    ~Bufs() {
        if (v) cudaFree(v);
        if (y) cudaFree(y);
        if (part) cudaFree(part);
        if (d) cudaFree(d);
    }
};

// out = M x (rows = true: m-vector from an n-vector) or M^T x (n-vector from an m-vector)
cudaError_t apply(const float* M, int64_t m, int64_t n, bool rows, const float* x, float* out, float* part,
                  int vec, cudaStream_t st) {
    if (rows) {
        rowdot_kernel<<<(unsigned)((m + kRowWarps - 1) / kRowWarps), 32 * kRowWarps, 0, st>>>(M, m, n, x, out, vec);
        return cudaGetLastError();
    }
    const int64_t nrb = (m + kColRows - 1) / kColRows;
    const int64_t cols_per_block = (int64_t)kColThreads * (vec ? 4 : 1);
    dim3 grid((unsigned)((n + cols_per_block - 1) / cols_per_block), (unsigned)nrb);
    coldot_partial_kernel<<<grid, kColThreads, 0, st>>>(M, m, n, x, part, vec);
    coldot_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nrb, n, out);
    return cudaGetLastError();
}

}  // namespace

// Host: the cubic of Eq. init_poly through (w, 1) and (z, 1), w = sqrt(f^2 - z^2),
// for ||X||_F = f (the paper's f = 1 polynomial of x / f). False when 2 z^2 <= f^2
// (the intervals [0, w] and [z, f] overlap) or w = 0.
bool init_cubic(double z, double f, double* a, double* b, double* w) {
    if (!(f > 0.0 && z > 0.0) || 2.0 * z * z <= f * f) return false;
    const double zn = std::min(z / f, 1.0);
    if (zn >= 1.0) return false;
    const double wn = std::sqrt(1.0 - zn * zn);
    const double den = zn * wn * (2.0 * zn * zn - 1.0);
    *a = (zn * zn * (zn + wn) - wn) / den / f;
    *b = (wn - zn) / den / (f * f * f);
    *w = f * wn;
    return true;
}

}  // namespace pe

extern "C" {

int pe_spectrum_bound(const void* X, int64_t m, int64_t n, const float* v0, int iters, double* z, double* f,
                      void* stream) {
    using namespace pe;
    if (!X || !v0 || !z || !f) return sfail(PE_EINVAL, "NULL argument");
    if (m < 1 || n < 1) return sfail(PE_EINVAL, "sizes must be >= 1");
    if (m > (1 << 20) || n > (1 << 20) || m * n > (int64_t)1 << 31)
        return sfail(PE_EINVAL, "matrix too large (m, n <= 2^20, m*n <= 2^31)");
    if (iters < 0 || iters > 10000) return sfail(PE_EINVAL, "iters must be in 0..10000");
    if (reinterpret_cast<uintptr_t>(X) % 4) return sfail(PE_EINVAL, "misaligned matrix pointer");
    const int64_t s = std::min(m, n);
    bool nz = false;
    for (int64_t i = 0; i < s; ++i) {
        if (!std::isfinite(v0[i])) return sfail(PE_EINVAL, "non-finite entry in v0");
        nz = nz || v0[i] != 0.f;
    }
    if (!nz) return sfail(PE_EINVAL, "v0 must be nonzero");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float* M = static_cast<const float*>(X);
    const bool short_rows = m <= n;   // X_0 is G (s = m) or G^T (s = n)
    const int64_t L = std::max(m, n);
    const int vec_rows = (n % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0) ? 1 : 0;
    const int64_t nrb = (m + kColRows - 1) / kColRows;
    const int64_t total = m * n;
    const int fblocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (total + 1023) / 1024));
    Bufs B;
    PE_SCU(cudaMalloc(&B.v, sizeof(float) * s));
    PE_SCU(cudaMalloc(&B.y, sizeof(float) * L));
    PE_SCU(cudaMalloc(&B.part, sizeof(float) * nrb * n));
    PE_SCU(cudaMalloc(&B.d, sizeof(double) * (3 + fblocks)));
    PE_SCU(cudaMemcpyAsync(B.v, v0, sizeof(float) * s, cudaMemcpyHostToDevice, st));
    // ||G||_F^2
    frob_partial_kernel<<<fblocks, 256, 0, st>>>(M, total, B.d + 3, vec_rows);
    sum_partials_kernel<<<1, 32, 0, st>>>(B.d + 3, fblocks, B.d);
    PE_SCU(cudaGetLastError());
    // unit start vector, then the power steps on G G^T (short rows) or G^T G
    sumsq_kernel<<<1, 1024, 0, st>>>(B.v, s, B.d + 1);
    scale_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(B.v, s, B.d + 1);
    PE_SCU(cudaGetLastError());
    for (int k = 0; k < iters; ++k) {
        // y = X_0^T v (up to the scale), v = X_0 y
        PE_SCU(apply(M, m, n, !short_rows, B.v, B.y, B.part, vec_rows, st));
        PE_SCU(apply(M, m, n, short_rows, B.y, B.v, B.part, vec_rows, st));
        sumsq_kernel<<<1, 1024, 0, st>>>(B.v, s, B.d + 1);
        scale_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(B.v, s, B.d + 1);
        PE_SCU(cudaGetLastError());
    }
    PE_SCU(apply(M, m, n, !short_rows, B.v, B.y, B.part, vec_rows, st));
    sumsq_kernel<<<1, 1024, 0, st>>>(B.y, L, B.d + 2);
    sumsq_kernel<<<1, 1024, 0, st>>>(B.v, s, B.d + 1);
    PE_SCU(cudaGetLastError());
    double h[3];
    PE_SCU(cudaMemcpyAsync(h, B.d, sizeof(h), cudaMemcpyDeviceToHost, st));
    PE_SCU(cudaStreamSynchronize(st));
    if (!std::isfinite(h[0]) || !std::isfinite(h[2])) return sfail(PE_ECUDA, "non-finite norm in the power method");
    const double nu = std::sqrt(h[0]);
    const double den = 1.01 * nu + 1e-7;
    *f = nu / den;
    // ||v|| = 1 up to rounding (0 when the iteration met the null space)
    *z = (h[1] > 0.0) ? std::sqrt(h[2] / h[1]) / den : 0.0;
    return PE_OK;
}

int pe_spectrum_aware_table_ex(double z, double f, double l, int T, double z_safety, unsigned flags, double* table,
                               double* info) {
    using namespace pe;
    if (!table) return sfail(PE_EINVAL, "table is NULL");
    if (!(l > 0.0 && l <= 1.0)) return sfail(PE_EINVAL, "l must be in (0, 1]");
    if (T < 0 || T + 1 > kMaxSteps) return sfail(PE_EINVAL, "T must be in 0..63");
    if (!std::isfinite(z) || !std::isfinite(f) || z < 0.0 || f < 0.0) return sfail(PE_EINVAL, "bad z or f");
    if (!(z_safety >= 0.0 && z_safety < 1.0)) return sfail(PE_EINVAL, "z_safety must be in [0, 1)");
    if (flags & ~(unsigned)PE_SPECTRUM_GATE) return sfail(PE_EINVAL, "unknown flags");
    const double zs = z * (1.0 - z_safety);
    double a = 0.0, b = 0.0, w = 0.0;
    const char* why = nullptr;
    // the plain composition with one more step, and its greedy bound after the last step
    std::vector<double> plain(3 * (T + 1)), pbounds(2 * (T + 2));
    int r = coeffs_table(5, l, T + 1, 1.01, -1.0, 0u, plain.data(), pbounds.data(), nullptr, &why);
    if (r != PE_OK) return sfail(r, why ? why : "coefficient solve failed");
    bool applied = init_cubic(zs, f, &a, &b, &w);
    double lp = l;
    if (applied) {
        // the cubic, then the composition for [l', 1]
        const double pf = f * (a + b * f * f);
        lp = std::min(l / w, pf);
        double l_final = lp;
        std::vector<double> rest(3 * std::max(T, 1)), rbounds(2 * (T + 1));
        if (T > 0) {
            r = coeffs_table(5, lp, T, 1.01, -1.0, 0u, rest.data(), rbounds.data(), nullptr, &why);
            if (r != PE_OK) return sfail(r, why ? why : "coefficient solve failed");
            l_final = rbounds[2 * T];
        }
        if (flags & PE_SPECTRUM_GATE) applied = l_final > pbounds[2 * (T + 1)];
        if (applied) {
            table[0] = a;
            table[1] = b;
            table[2] = 0.0;
            for (int k = 0; k < 3 * T; ++k) table[3 + k] = rest[k];
        }
    }
    if (!applied) {
        lp = l;
        for (int k = 0; k < 3 * (T + 1); ++k) table[k] = plain[k];
    }
    if (info) {
        info[0] = applied ? 1.0 : 0.0;
        info[1] = zs;
        info[2] = f;
        info[3] = a;
        info[4] = b;
        info[5] = lp;
    }
    return PE_OK;
}

int pe_spectrum_aware_table(double z, double f, double l, int T, double* table, double* info) {
    return pe_spectrum_aware_table_ex(z, f, l, T, 0.0, 0u, table, info);
}

int pe_polar_spectrum_aware_ex(void* X, int64_t m, int64_t n, double l, int T, int dtype, const float* v0, int iters,
                               double z_safety, unsigned flags, double* info, void* stream) {
    using namespace pe;
    if (dtype != PE_FP32 && dtype != PE_BF16 && dtype != PE_BF16X3) return sfail(PE_EINVAL, "bad dtype");
    if (T < 0 || T + 1 > kMaxSteps) return sfail(PE_EINVAL, "T must be in 0..63");
    if (!(l > 0.0 && l <= 1.0)) return sfail(PE_EINVAL, "l must be in (0, 1]");
    if (!(z_safety >= 0.0 && z_safety < 1.0)) return sfail(PE_EINVAL, "z_safety must be in [0, 1)");
    if (flags & ~(unsigned)PE_SPECTRUM_GATE) return sfail(PE_EINVAL, "unknown flags");
    double z = 0.0, f = 0.0;
    int r = pe_spectrum_bound(X, m, n, v0, iters, &z, &f, stream);
    if (r != PE_OK) return r;
    std::vector<double> table(3 * (T + 1));
    double inf[6];
    r = pe_spectrum_aware_table_ex(z, f, l, T, z_safety, flags, table.data(), inf);
    if (r != PE_OK) return r;
    if (info)
        for (int k = 0; k < 6; ++k) info[k] = inf[k];
    return pe_polar(X, m, n, table.data(), T + 1, dtype, stream);
}

int pe_polar_spectrum_aware(void* X, int64_t m, int64_t n, double l, int T, int dtype, const float* v0, int iters,
                            double* info, void* stream) {
    return pe_polar_spectrum_aware_ex(X, m, n, l, T, dtype, v0, iters, pe::kZSafetyFp32, 0u, info, stream);
}

}  // extern "C"
